// lmood_api.cu -- C ABI of the library (declared in include/lmood.h): mesh set-up (node ->
// corner adjacency, boundary-condition resolution), state buffers, and the host
// side of the step (kernel sequence and the MOOD loop over compacted lists).
#include <algorithm>
#include <chrono>
#include <array>
#include <functional>
#include <cmath>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "lmood_internal.h"

using namespace lmood;

namespace {

thread_local std::string g_err;

template <class T> lmood_status upload(DevAllocs &A, T **dst, const T *src, size_t n, cudaStream_t st) {
    lmood_status s = A.alloc((void **)dst, n * sizeof(T));
    if (s) return s;
    if (n && src) LM_CUDA(cudaMemcpyAsync(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice, st));
    return LMOOD_OK;
}

void parallel_for(int64_t n, const std::function<void(int64_t, int64_t)> &fn) {
    unsigned nt = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
    if (n < 20000) nt = 1;
    std::vector<std::thread> th;
    const int64_t chunk = (n + nt - 1) / nt;
    for (unsigned t = 0; t < nt; ++t) {
        const int64_t b = t * chunk, e = std::min<int64_t>(n, b + chunk);
        if (b < e) th.emplace_back(fn, b, e);
    }
    for (auto &t : th) t.join();
}

}  // namespace

lmood_status lmood::fail(lmood_status st, const std::string &msg) {
    g_err = msg;
    return st;
}

// error message setter shared with the other translation units of the library
void lmood_internal_set_error(const char *msg) { g_err = msg; }

// =======================================================================================
// mesh
// =======================================================================================

static double host_volume(int d, const double *x, int64_t np, const int32_t *c2n, int64_t nc, int64_t c) {
    int p[4];
    for (int k = 0; k <= d; ++k) p[k] = c2n[k * nc + c];
    auto X = [&](int k, int a) { return x[a * np + p[k]]; };
    if (d == 2) return 0.5 * ((X(1, 0) - X(0, 0)) * (X(2, 1) - X(0, 1)) - (X(1, 1) - X(0, 1)) * (X(2, 0) - X(0, 0)));
    double e[3][3];
    for (int k = 0; k < 3; ++k)
        for (int a = 0; a < 3; ++a) e[k][a] = X(k + 1, a) - X(0, a);
    return (e[0][0] * (e[1][1] * e[2][2] - e[1][2] * e[2][1]) - e[0][1] * (e[1][0] * e[2][2] - e[1][2] * e[2][0]) +
            e[0][2] * (e[1][0] * e[2][1] - e[1][1] * e[2][0])) /
           6.0;
}

extern "C" lmood_status lmood_params_default(int dim, lmood_params *p) {
    if (!p || (dim != 2 && dim != 3)) return fail(LMOOD_ERR_ARG, "lmood_params_default: bad dim or NULL");
    std::memset(p, 0, sizeof(*p));
    p->cfl = dim == 2 ? 0.4 : 0.25;
    p->Cv = 0.2;
    p->Ci = 0.1;
    p->delta0 = 1e-4;
    p->delta1 = 1e-3;
    p->dt_fixed = 0.0;
    p->max_mood_iters = 100000;
    p->order = 2;
    p->mood = 1;
    p->graph = 1;
    p->cascade = 2;
    return LMOOD_OK;
}

// Per-node boundary conditions from the face tags (Appendix B). The velocity subspace:
// strongest first, clamped > slip > free (k distinct slip planes leave their intersection);
// nodes touched by a traction, pressure or prescribed-velocity face get BC_EXT (their forces
// and constraint act in the nodal solve). Faces are [dim][nb], oriented outward.
static lmood_status resolve_bcs(int dim, int64_t Np, int64_t n_bfaces, const double *x, const int *bface,
                                const int *btag, std::vector<unsigned char> &ndof, std::vector<double> &bct,
                                bool &has_ext) {
    ndof.assign(Np, (unsigned char)dim);
    bct.assign(6 * Np, 0.0);
    has_ext = false;
    std::vector<unsigned char> clamped(Np, 0), ext(Np, 0);
    std::vector<std::vector<std::array<double, 3>>> planes(Np);
    for (int64_t f = 0; f < n_bfaces; ++f) {
        int q[3];
        for (int a = 0; a < dim; ++a) q[a] = bface[a * n_bfaces + f];
        std::array<double, 3> nrm{0, 0, 0};
        if (dim == 2) {
            nrm[0] = x[1 * Np + q[1]] - x[1 * Np + q[0]];
            nrm[1] = x[0 * Np + q[0]] - x[0 * Np + q[1]];
        } else {
            double u[3], w[3];
            for (int a = 0; a < 3; ++a) {
                u[a] = x[a * Np + q[1]] - x[a * Np + q[0]];
                w[a] = x[a * Np + q[2]] - x[a * Np + q[0]];
            }
            nrm = {u[1] * w[2] - u[2] * w[1], u[2] * w[0] - u[0] * w[2], u[0] * w[1] - u[1] * w[0]};
        }
        const double len = std::sqrt(nrm[0] * nrm[0] + nrm[1] * nrm[1] + nrm[2] * nrm[2]);
        if (!(len > 0)) return fail(LMOOD_ERR_MESH, "degenerate boundary face");
        for (double &v : nrm) v /= len;
        for (int a = 0; a < dim; ++a) {
            const int p = q[a];
            if (btag[f] == TAG_CLAMPED) clamped[p] = 1;
            if (btag[f] >= TAG_TRACTION) {
                ext[p] |= btag[f] == TAG_CONTACT ? 2 : 1;
                has_ext = true;
            }
            if (btag[f] != TAG_SLIP) continue;
            bool known = false;
            for (auto &pl : planes[p])
                if (std::fabs(pl[0] * nrm[0] + pl[1] * nrm[1] + pl[2] * nrm[2]) > 1.0 - 1e-12) known = true;
            if (!known) planes[p].push_back(nrm);
        }
    }
    for (int64_t p = 0; p < Np; ++p) {
        const int k = clamped[p] ? dim : (int)planes[p].size();
        auto T = [&](int i, int a) -> double & { return bct[(i * 3 + a) * Np + p]; };
        if (k >= dim) {
            ndof[p] = 0;
        } else if (k > 0) {
            const auto &n1 = planes[p][0];
            if (dim == 2) {  // one wall line: the free direction is its tangent
                ndof[p] = 1;
                T(0, 0) = n1[1];
                T(0, 1) = -n1[0];
            } else if (k == 1) {  // one wall plane: Gram-Schmidt of the two axes least aligned with n
                int ax[3] = {0, 1, 2};
                std::sort(ax, ax + 3, [&](int i, int j) { return std::fabs(n1[i]) < std::fabs(n1[j]); });
                double t1[3] = {0, 0, 0};
                t1[ax[0]] = 1.0;
                const double dn = t1[0] * n1[0] + t1[1] * n1[1] + t1[2] * n1[2];
                for (int a = 0; a < 3; ++a) t1[a] -= dn * n1[a];
                const double l1 = std::sqrt(t1[0] * t1[0] + t1[1] * t1[1] + t1[2] * t1[2]);
                for (int a = 0; a < 3; ++a) t1[a] /= l1;
                double t2[3] = {n1[1] * t1[2] - n1[2] * t1[1], n1[2] * t1[0] - n1[0] * t1[2], n1[0] * t1[1] - n1[1] * t1[0]};
                const double l2 = std::sqrt(t2[0] * t2[0] + t2[1] * t2[1] + t2[2] * t2[2]);
                for (int a = 0; a < 3; ++a) {
                    T(0, a) = t1[a];
                    T(1, a) = t2[a] / l2;
                }
                ndof[p] = 2;
            } else {  // two wall planes: their intersection line
                const auto &n2 = planes[p][1];
                double l[3] = {n1[1] * n2[2] - n1[2] * n2[1], n1[2] * n2[0] - n1[0] * n2[2], n1[0] * n2[1] - n1[1] * n2[0]};
                const double ll = std::sqrt(l[0] * l[0] + l[1] * l[1] + l[2] * l[2]);
                for (int a = 0; a < 3; ++a) T(0, a) = l[a] / ll;
                ndof[p] = 1;
            }
        }
        if (ext[p] & 1) ndof[p] |= BC_EXT;
        if (ext[p] & 2) ndof[p] |= BC_CONTACT;
    }
    return LMOOD_OK;
}

extern "C" lmood_status lmood_mesh_create(int dim, int64_t n_nodes, const double *x, int64_t n_cells,
                                          const int32_t *c2n, int64_t n_bfaces, const int32_t *bface,
                                          const int32_t *btag, const int32_t *cell_inst, int32_t n_inst,
                                          void *stream, lmood_mesh *out) {
    if (!out) return fail(LMOOD_ERR_ARG, "lmood_mesh_create: out is NULL");
    *out = nullptr;
    if (dim != 2 && dim != 3) return fail(LMOOD_ERR_ARG, "lmood_mesh_create: dim must be 2 or 3");
    if (n_nodes <= 0 || n_cells <= 0 || !x || !c2n) return fail(LMOOD_ERR_ARG, "lmood_mesh_create: empty mesh or NULL array");
    const int nv = dim + 1;
    // the kernels index with 32-bit integers: the largest offsets are those of the corner
    // matrices (NS (D+1) N), of F (D^2 N) and of the node moments (NMOM Np)
    {
        const int64_t ns = dim * (dim + 1) / 2, nmom = (dim == 2 ? ops_dim2() : ops_dim3()).nmom;
        if (n_cells > INT32_MAX / (ns * nv) || n_cells > INT32_MAX / (dim * dim) || n_nodes > INT32_MAX / nmom)
            return fail(LMOOD_ERR_ARG, "lmood_mesh_create: mesh too large for 32-bit indices (at most " +
                                           std::to_string(INT32_MAX / (ns * nv)) + " cells and " +
                                           std::to_string(INT32_MAX / nmom) + " nodes in " + std::to_string(dim) + "D)");
    }
    if (n_bfaces < 0 || (n_bfaces > 0 && (!bface || !btag))) return fail(LMOOD_ERR_ARG, "lmood_mesh_create: boundary faces");
    if (cell_inst ? n_inst < 1 : n_inst > 1) return fail(LMOOD_ERR_ARG, "lmood_mesh_create: bad instance count");
    if (!cell_inst) n_inst = 1;
    const int64_t N = n_cells, Np = n_nodes;
    // validation: indices and orientation
    for (int64_t i = 0; i < N * nv; ++i)
        if (c2n[i] < 0 || c2n[i] >= Np) return fail(LMOOD_ERR_MESH, "lmood_mesh_create: node index out of range in c2n");
    for (int64_t c = 0; c < N; ++c)
        if (!(host_volume(dim, x, Np, c2n, N, c) > 0.0))
            return fail(LMOOD_ERR_MESH, "lmood_mesh_create: cell " + std::to_string(c) + " has non-positive volume");
    for (int64_t i = 0; i < n_bfaces * dim; ++i)
        if (bface[i] < 0 || bface[i] >= Np) return fail(LMOOD_ERR_MESH, "lmood_mesh_create: node index out of range in bface");
    for (int64_t i = 0; i < n_bfaces; ++i)
        if (btag[i] < 0 || btag[i] > 6) return fail(LMOOD_ERR_ARG, "lmood_mesh_create: boundary tag must be 0 to 6");
    std::vector<int> node_inst;
    if (cell_inst) {
        node_inst.assign(Np, -1);
        for (int64_t c = 0; c < N; ++c) {
            const int ci = cell_inst[c];
            if (ci < 0 || ci >= n_inst) return fail(LMOOD_ERR_ARG, "lmood_mesh_create: cell instance out of range");
            for (int k = 0; k < nv; ++k) {
                int &ni = node_inst[c2n[k * N + c]];
                if (ni >= 0 && ni != ci) return fail(LMOOD_ERR_MESH, "lmood_mesh_create: a node is shared by two instances");
                ni = ci;
            }
        }
    }
    // node -> corner CSR: corners of each node in ascending cell id; corner id = k N + c
    std::vector<int> off(Np + 1, 0), n2c(N * nv);
    for (int64_t c = 0; c < N; ++c)
        for (int k = 0; k < nv; ++k) off[c2n[k * N + c] + 1]++;
    for (int64_t p = 0; p < Np; ++p) off[p + 1] += off[p];
    int max_deg = 0;
    for (int64_t p = 0; p < Np; ++p) max_deg = std::max(max_deg, off[p + 1] - off[p]);
    {
        std::vector<int> pos(off.begin(), off.end() - 1);
        for (int64_t c = 0; c < N; ++c)
            for (int k = 0; k < nv; ++k) n2c[pos[c2n[k * N + c]]++] = (int)(k * N + c);
    }
    // the nodes of each window of 256 consecutive ones in order of their cell count (stable),
    // so that the per-node kernels give a warp nodes with equally long loops while a block
    // still reads the cells of one neighbourhood
    std::vector<int> perm(Np);
    {
        constexpr int64_t kWin = 256;
        std::vector<int64_t> first(max_deg + 2);
        for (int64_t w0 = 0; w0 < Np; w0 += kWin) {
            const int64_t w1 = std::min(Np, w0 + kWin);
            std::fill(first.begin(), first.end(), 0);
            for (int64_t p = w0; p < w1; ++p) first[off[p + 1] - off[p] + 1]++;
            first[0] = w0;
            for (int d2 = 0; d2 <= max_deg; ++d2) first[d2 + 1] += first[d2];
            for (int64_t p = w0; p < w1; ++p) perm[first[off[p + 1] - off[p]]++] = (int)p;
        }
    }
    // (node, neighbour) pairs of the least-squares sums: sum_p deg(p) (deg(p) - 1)
    int64_t nnz = 0;
    for (int64_t p = 0; p < Np; ++p) nnz += (int64_t)(off[p + 1] - off[p]) * (off[p + 1] - off[p] - 1);
    // boundary faces: oriented outward (the area vector points away from the vertex of the
    // face's cell that is not on the face), tags, the faces around each node
    std::vector<int> bf(bface, bface + n_bfaces * dim), tags(btag, btag + n_bfaces);
    for (int64_t f = 0; f < n_bfaces; ++f) {
        int q[3];
        for (int a = 0; a < dim; ++a) q[a] = bf[a * n_bfaces + f];
        int opp = -1, owners = 0;  // the cells having the face: exactly one for a boundary face
        for (int j = off[q[0]]; j < off[q[0] + 1]; ++j) {
            const int64_t c = n2c[j] % N;
            int hits = 0, other = -1;
            for (int k = 0; k < nv; ++k) {
                const int r = c2n[k * N + c];
                bool on = false;
                for (int a = 0; a < dim; ++a) on |= r == q[a];
                if (on) ++hits;
                else other = r;
            }
            if (hits == dim) {
                if (owners++ == 0) opp = other;
            }
        }
        if (owners != 1)
            return fail(LMOOD_ERR_MESH, "lmood_mesh_create: boundary face " + std::to_string(f) + " is a face of " +
                                            std::to_string(owners) + " cells (a boundary face belongs to exactly one)");
        double nrm[3] = {0, 0, 0};
        if (dim == 2) {
            nrm[0] = x[1 * Np + q[1]] - x[1 * Np + q[0]];
            nrm[1] = x[0 * Np + q[0]] - x[0 * Np + q[1]];
        } else {
            double u[3], w[3];
            for (int a = 0; a < 3; ++a) {
                u[a] = x[a * Np + q[1]] - x[a * Np + q[0]];
                w[a] = x[a * Np + q[2]] - x[a * Np + q[0]];
            }
            nrm[0] = u[1] * w[2] - u[2] * w[1];
            nrm[1] = u[2] * w[0] - u[0] * w[2];
            nrm[2] = u[0] * w[1] - u[1] * w[0];
        }
        double dot = 0.0;
        for (int a = 0; a < dim; ++a) {
            double xf = 0.0;
            for (int i = 0; i < dim; ++i) xf += x[a * Np + q[i]];
            dot += nrm[a] * (xf / dim - x[a * Np + opp]);
        }
        if (dot < 0.0) std::swap(bf[0 * n_bfaces + f], bf[1 * n_bfaces + f]);
    }
    // a face listed twice (in any node order) would give its nodes its traction, pressure or
    // velocity share twice
    {
        std::vector<std::array<int, 4>> keys(n_bfaces);
        for (int64_t f = 0; f < n_bfaces; ++f) {
            std::array<int, 4> k{-1, -1, -1, (int)f};
            for (int a = 0; a < dim; ++a) k[a] = bf[a * n_bfaces + f];
            std::sort(k.begin(), k.begin() + dim);
            keys[f] = k;
        }
        std::sort(keys.begin(), keys.end());
        for (int64_t i = 1; i < n_bfaces; ++i)
            if (std::equal(keys[i].begin(), keys[i].begin() + 3, keys[i - 1].begin()))
                return fail(LMOOD_ERR_MESH, "lmood_mesh_create: boundary faces " + std::to_string(keys[i - 1][3]) +
                                                " and " + std::to_string(keys[i][3]) + " are the same face");
    }
    std::vector<int> nbf_off(Np + 1, 0), nbf_idx(n_bfaces * dim);
    for (int64_t f = 0; f < n_bfaces; ++f)
        for (int a = 0; a < dim; ++a) nbf_off[bf[a * n_bfaces + f] + 1]++;
    for (int64_t p = 0; p < Np; ++p) nbf_off[p + 1] += nbf_off[p];
    {
        std::vector<int> pos(nbf_off.begin(), nbf_off.end() - 1);
        for (int64_t f = 0; f < n_bfaces; ++f)
            for (int a = 0; a < dim; ++a) nbf_idx[pos[bf[a * n_bfaces + f]]++] = (int)f;
    }
    std::vector<unsigned char> ndof;
    std::vector<double> bct;
    bool has_ext = false;
    {
        lmood_status r = resolve_bcs(dim, Np, n_bfaces, x, bf.data(), tags.data(), ndof, bct, has_ext);
        if (r) return fail(r, std::string("lmood_mesh_create: ") + lmood_last_error());
    }
    // device copies
    cudaStream_t st = (cudaStream_t)stream;
    auto *m = new lmood_mesh_s();
    m->dim = dim;
    m->n_inst = n_inst;
    m->np = Np;
    m->nc = N;
    m->st_nnz = nnz;
    m->max_deg = max_deg;
    m->st = st;
    m->ops = dim == 2 ? &ops_dim2() : &ops_dim3();
    Geo &g = m->geo;
    g.N = (int)N;
    g.Np = (int)Np;
    g.n_inst = n_inst;
    lmood_status s;
    int *d_c2n, *d_off, *d_n2c, *d_perm, *d_ci = nullptr, *d_ni = nullptr;
    unsigned char *d_nd;
    double *d_bt;
    std::vector<int> c2n_i(c2n, c2n + N * nv);
    if ((s = upload(m->mem, &d_c2n, c2n_i.data(), c2n_i.size(), st)) ||
        (s = upload(m->mem, &d_off, off.data(), off.size(), st)) ||
        (s = upload(m->mem, &d_n2c, n2c.data(), n2c.size(), st)) ||
        (s = upload(m->mem, &d_perm, perm.data(), perm.size(), st)) ||
        (s = upload(m->mem, &d_nd, ndof.data(), ndof.size(), st)) ||
        (s = upload(m->mem, &d_bt, bct.data(), bct.size(), st)) ||
        (s = upload(m->mem, &m->x0, x, (size_t)(dim * Np), st))) {
        m->mem.release();
        delete m;
        return s;
    }
    if (cell_inst) {
        std::vector<int> ci(cell_inst, cell_inst + N);
        if ((s = upload(m->mem, &d_ci, ci.data(), ci.size(), st)) ||
            (s = upload(m->mem, &d_ni, node_inst.data(), node_inst.size(), st))) {
            m->mem.release();
            delete m;
            return s;
        }
    }
    g.c2n = d_c2n;
    g.n2c_off = d_off;
    g.n2c = d_n2c;
    g.node_perm = d_perm;
    g.bc_ndof = d_nd;
    g.bc_t = d_bt;
    g.cell_inst = d_ci;
    g.node_inst = d_ni;
    m->d_ndof = d_nd;
    m->d_bct = d_bt;
    m->nb = n_bfaces;
    m->has_ext = has_ext;
    m->h_x0.assign(x, x + dim * Np);
    m->h_bf = bf;
    m->h_btag = tags;
    g.nbf = (int)n_bfaces;
    {
        std::vector<double> c0(2 + 2 * 3 * kMaxContact, 0.0);  // no contact walls
        if ((s = upload(m->mem, &m->d_contact, c0.data(), c0.size(), st))) {
            m->mem.release();
            delete m;
            return s;
        }
        g.contact = m->d_contact;
    }
    if (n_bfaces > 0) {
        int *d_bfn, *d_noff, *d_nidx;
        std::vector<unsigned char> t8(tags.begin(), tags.end());
        std::vector<double> zeros((size_t)dim * n_bfaces, 0.0);
        if ((s = upload(m->mem, &d_bfn, bf.data(), bf.size(), st)) ||
            (s = upload(m->mem, &m->d_btag, t8.data(), t8.size(), st)) ||
            (s = upload(m->mem, &m->d_bfval, zeros.data(), zeros.size(), st)) ||
            (s = upload(m->mem, &d_noff, nbf_off.data(), nbf_off.size(), st)) ||
            (s = upload(m->mem, &d_nidx, nbf_idx.data(), nbf_idx.size(), st))) {
            m->mem.release();
            delete m;
            return s;
        }
        g.bf_nodes = d_bfn;
        g.bf_tag = m->d_btag;
        g.bf_val = m->d_bfval;
        g.nbf_off = d_noff;
        g.nbf_idx = d_nidx;
    }
    cudaError_t e = cudaStreamSynchronize(st);  // host vectors die at return
    if (e != cudaSuccess) {
        m->mem.release();
        delete m;
        return fail(LMOOD_ERR_CUDA, std::string("lmood_mesh_create: ") + cudaGetErrorString(e));
    }
    *out = m;
    return LMOOD_OK;
}

extern "C" lmood_status lmood_mesh_destroy(lmood_mesh m) {
    if (!m) return fail(LMOOD_ERR_ARG, "lmood_mesh_destroy: NULL");
    cudaStreamSynchronize(m->st);
    for (lmood_state s : m->states) {  // destroyed out of order: the states can only be destroyed now
        s->M = nullptr;
        s->broken = true;
    }
    m->mem.release();
    delete m;
    return LMOOD_OK;
}

extern "C" lmood_status lmood_mesh_info(lmood_mesh m, int64_t *o) {
    if (!m || !o) return fail(LMOOD_ERR_ARG, "lmood_mesh_info: NULL");
    o[0] = m->np;
    o[1] = m->nc;
    o[2] = m->dim;
    o[3] = m->st_nnz;
    o[4] = m->max_deg;
    o[5] = m->n_inst;
    return LMOOD_OK;
}

extern "C" lmood_status lmood_mesh_set_bc_values(lmood_mesh m, const double *values, int is_device) {
    if (!m || !values) return fail(LMOOD_ERR_ARG, "lmood_mesh_set_bc_values: NULL argument");
    if (m->nb == 0) return LMOOD_OK;
    LM_CUDA(cudaMemcpyAsync(m->d_bfval, values, (size_t)m->dim * m->nb * sizeof(double),
                            is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, m->st));
    if (!is_device) LM_CUDA(cudaStreamSynchronize(m->st));
    ++m->bc_version;
    return LMOOD_OK;
}

extern "C" lmood_status lmood_mesh_set_contact(lmood_mesh m, int n_planes, const double *planes, double eps) {
    if (!m || n_planes < 0 || n_planes > kMaxContact || (n_planes > 0 && !planes) || !(eps >= 0.0))
        return fail(LMOOD_ERR_ARG, "lmood_mesh_set_contact: bad argument (at most 4 planes, eps >= 0)");
    const int D = m->dim;
    std::vector<double> c(2 + 2 * 3 * kMaxContact, 0.0);
    c[0] = n_planes;
    c[1] = eps;
    for (int k = 0; k < n_planes; ++k) {
        double nn = 0.0;
        for (int a = 0; a < D; ++a) nn += planes[k * 2 * D + D + a] * planes[k * 2 * D + D + a];
        if (!(std::fabs(nn - 1.0) <= 1e-12)) return fail(LMOOD_ERR_ARG, "lmood_mesh_set_contact: normals must be unit vectors");
        for (int i = 0; i < 2 * D; ++i) c[2 + 2 * D * k + i] = planes[k * 2 * D + i];
    }
    LM_CUDA(cudaMemcpyAsync(m->d_contact, c.data(), c.size() * sizeof(double), cudaMemcpyHostToDevice, m->st));
    LM_CUDA(cudaStreamSynchronize(m->st));
    ++m->bc_version;
    return LMOOD_OK;
}

extern "C" lmood_status lmood_mesh_set_btag(lmood_mesh m, const int32_t *btag) {
    if (!m || (!btag && m->nb > 0)) return fail(LMOOD_ERR_ARG, "lmood_mesh_set_btag: NULL argument");
    for (int64_t f = 0; f < m->nb; ++f)
        if (btag[f] < 0 || btag[f] > 6) return fail(LMOOD_ERR_ARG, "lmood_mesh_set_btag: boundary tag must be 0 to 6");
    std::vector<int> tags(btag, btag + m->nb);
    std::vector<unsigned char> ndof;
    std::vector<double> bct;
    bool has_ext = false;
    lmood_status r = resolve_bcs(m->dim, m->np, m->nb, m->h_x0.data(), m->h_bf.data(), tags.data(), ndof, bct, has_ext);
    if (r) return fail(r, std::string("lmood_mesh_set_btag: ") + lmood_last_error());
    // in place: graphs captured on this mesh stay valid
    LM_CUDA(cudaMemcpyAsync(m->d_ndof, ndof.data(), ndof.size(), cudaMemcpyHostToDevice, m->st));
    LM_CUDA(cudaMemcpyAsync(m->d_bct, bct.data(), bct.size() * sizeof(double), cudaMemcpyHostToDevice, m->st));
    std::vector<unsigned char> t8(tags.begin(), tags.end());
    if (m->nb > 0) LM_CUDA(cudaMemcpyAsync(m->d_btag, t8.data(), t8.size(), cudaMemcpyHostToDevice, m->st));
    LM_CUDA(cudaStreamSynchronize(m->st));
    m->h_btag = tags;
    m->has_ext = has_ext;
    ++m->bc_version;
    return LMOOD_OK;
}

// =======================================================================================
// state
// =======================================================================================
static constexpr int kMaxPending = 64;

static void timing_drain(lmood_state s) {
    for (size_t i = 0; i < s->pend_cls.size(); ++i) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, s->ev[2 * i], s->ev[2 * i + 1]) == cudaSuccess) s->kms[s->pend_cls[i]] += ms;
    }
    s->pend_cls.clear();
}

// Launch helper: counts the launch and, with timing on, brackets it with a pair of events.
template <class F> static void timed(lmood_state s, int cls, int n_launch, F &&launch) {
    s->klaunch[cls] += n_launch;
    if (!s->timing || s->pend_cls.size() >= (size_t)kMaxPending) {
        launch();
        return;
    }
    const size_t i = s->pend_cls.size();
    cudaEventRecord(s->ev[2 * i], s->M->st);
    launch();
    cudaEventRecord(s->ev[2 * i + 1], s->M->st);
    s->pend_cls.push_back(cls);
}

void lmood::swap_state(lmood_state s) {
    s->parity ^= 1;
    Fld &f = s->f;
    std::swap(f.x, f.x1);
    std::swap(f.vp, f.vp1);
    std::swap(f.v, f.v1);
    std::swap(f.e, f.e1);
    std::swap(f.F, f.F1);
    std::swap(f.xc, f.xc1);
    std::swap(f.rho, f.rho1);
    std::swap(s->tau, f.tau1);
    std::swap(f.z, f.z1);
    std::swap(f.gf, f.gf1);
    double *dt = const_cast<double *>(f.dt);
    f.dt = (const double *)f.dtn;
    f.dtn = (unsigned long long *)dt;
}

static Prm kernel_params(const lmood_params &p, const lmood_material &m) {
    Prm k{};
    k.cfl = p.cfl;
    k.Cv = p.Cv;
    k.Ci = p.Ci;
    k.delta0 = p.delta0;
    k.delta1 = p.delta1;
    k.dt_fixed = p.dt_fixed;
    k.lam = m.lambda;
    k.irho0 = 1.0 / m.rho0;
    k.shear_a = m.shear_a;
    k.eos = m.eos;
    k.gamma = m.gamma;
    k.pinf = m.p_inf;
    k.p0 = m.p0;
    k.rho0 = m.rho0;
    k.base_order = p.order == 1 ? 1 : 2;
    k.mood = p.mood ? 1 : 0;
    k.vol_coeff = m.vol_coeff ? 1 : 0;
    k.cascade = p.cascade == 3 ? 3 : 2;
    return k;
}

static void state_free(lmood_state s) {
    tapes_orphan(s);
    if (s->M) {
        cudaStreamSynchronize(s->M->st);
        auto &v = s->M->states;
        v.erase(std::remove(v.begin(), v.end(), s), v.end());
    }
    for (cudaEvent_t e : s->ev) cudaEventDestroy(e);
    for (int p = 0; p < 2; ++p) {
        if (s->gexec[p]) cudaGraphExecDestroy(s->gexec[p]);
        if (s->graph[p]) cudaGraphDestroy(s->graph[p]);
        if (s->cexec[p]) cudaGraphExecDestroy(s->cexec[p]);
        if (s->cgraph[p]) cudaGraphDestroy(s->cgraph[p]);
        for (cudaEvent_t e : s->gev[p])
            if (e) cudaEventDestroy(e);
    }
    if (s->h_run) cudaFreeHost(s->h_run);
    if (s->body_st) cudaStreamDestroy(s->body_st);
    if (s->cap_st) cudaStreamDestroy(s->cap_st);
    if (s->aux_st) cudaStreamDestroy(s->aux_st);
    for (cudaEvent_t e : s->set_ev)
        if (e) cudaEventDestroy(e);
    if (s->h_report) cudaFreeHost(s->h_report);
    s->mem.release();
    if (s->h_cnt) cudaFreeHost(s->h_cnt);
    if (s->h_dt) cudaFreeHost(s->h_dt);
    delete s;
}

extern "C" lmood_status lmood_state_destroy(lmood_state s) {
    if (!s) return fail(LMOOD_ERR_ARG, "lmood_state_destroy: NULL");
    state_free(s);
    return LMOOD_OK;
}

lmood_status lmood::sync_check(lmood_state s, const char *where) {
    cudaError_t e = cudaStreamSynchronize(s->M->st);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
        s->broken = true;
        return fail(LMOOD_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
    }
    return LMOOD_OK;
}

// counts the entries of mu that are not > 0 (NaN included) into *bad
__global__ static void k_count_nonpositive(const double *mu, int64_t n, int *bad) {
    int k = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        k += !(mu[i] > 0.0);
    if (k) atomicAdd(bad, k);
}

static lmood_status state_init(lmood_mesh M, const lmood_material *mat, const double *mu_cell, const double *v_cell,
                               const double *F_cell, const lmood_params *prm, lmood_state *out, bool dev);

extern "C" lmood_status lmood_state_init(lmood_mesh M, const lmood_material *mat, const double *mu_cell,
                                         const double *v_cell, const double *F_cell, const lmood_params *prm,
                                         lmood_state *out) {
    return state_init(M, mat, mu_cell, v_cell, F_cell, prm, out, false);
}

extern "C" lmood_status lmood_state_init_device(lmood_mesh M, const lmood_material *mat, const double *mu_cell,
                                                const double *v_cell, const double *F_cell, const lmood_params *prm,
                                                lmood_state *out) {
    return state_init(M, mat, mu_cell, v_cell, F_cell, prm, out, true);
}

static lmood_status state_init(lmood_mesh M, const lmood_material *mat, const double *mu_cell, const double *v_cell,
                               const double *F_cell, const lmood_params *prm, lmood_state *out, bool dev) {
    if (!out) return fail(LMOOD_ERR_ARG, "lmood_state_init: out is NULL");
    *out = nullptr;
    if (!M || !mat || !mu_cell || !v_cell || !prm) return fail(LMOOD_ERR_ARG, "lmood_state_init: NULL argument");
    if (!(mat->rho0 > 0)) return fail(LMOOD_ERR_ARG, "lmood_state_init: rho0 must be positive");
    if (!(mat->shear_a >= -1.0 && mat->shear_a <= 0.5))
        return fail(LMOOD_ERR_ARG, "lmood_state_init: shear_a must lie in [-1, 1/2]");
    if (mat->eos != 0 && !(mat->eos == 1 && mat->gamma > 1.0 && mat->p0 + mat->p_inf > 0.0))
        return fail(LMOOD_ERR_ARG, "lmood_state_init: eos must be 0, or 1 with gamma > 1 and p0 + p_inf > 0");
    if (prm->graph < 0 || prm->graph > 3 || (prm->graph == 2 && (mat->shear_a != -1.0 || mat->eos != 0)))
        return fail(LMOOD_ERR_ARG, "lmood_state_init: graph must be 0, 1, 2 or 3 (2: neo-Hookean material only)");
    if (!(prm->cfl > 0) || prm->max_mood_iters < 0 || (prm->order != 1 && prm->order != 2) ||
        (prm->cascade != 2 && prm->cascade != 3))
        return fail(LMOOD_ERR_ARG, "lmood_state_init: bad parameters");
    const int D = M->dim, NV = D + 1, NS = D * (D + 1) / 2;
    const int64_t N = M->nc, Np = M->np;
    if (!dev)
        for (int64_t c = 0; c < N; ++c)
            if (!(mu_cell[c] > 0)) return fail(LMOOD_ERR_ARG, "lmood_state_init: mu must be positive");
    auto *s = new lmood_state_s();
    s->M = M;
    s->prm = *prm;
    s->mat = *mat;
    s->kp = kernel_params(*prm, *mat);
    cudaStream_t st = M->st;
    Fld &f = s->f;
    lmood_status r = LMOOD_OK;
    auto A = [&](void **p, size_t bytes) {
        if (r == LMOOD_OK) r = s->mem.alloc(p, bytes);
    };
    const size_t nd = sizeof(double);
    A((void **)&f.x, D * Np * nd);
    A((void **)&f.x1, D * Np * nd);
    A((void **)&f.vp, D * Np * nd);
    A((void **)&f.vp1, D * Np * nd);
    A((void **)&f.vs, D * Np * nd);
    A((void **)&f.v, D * N * nd);
    A((void **)&f.v1, D * N * nd);
    A((void **)&f.e, N * nd);
    A((void **)&f.e1, N * nd);
    A((void **)&f.F, D * D * N * nd);
    A((void **)&f.F1, D * D * N * nd);
    A((void **)&f.xc, D * N * nd);
    A((void **)&f.xc1, D * N * nd);
    A((void **)&f.rho, N * nd);
    A((void **)&f.rho1, N * nd);
    A((void **)&s->tau, N * nd);
    A((void **)&f.tau1, N * nd);
    A((void **)&s->m, N * nd);
    A((void **)&s->im, N * nd);
    A((void **)&f.z, N * nd);
    A((void **)&f.z1, N * nd);
    A((void **)&f.mom, (size_t)M->ops->nmom * Np * nd);
    A((void **)&f.rlo, Np * nd);
    A((void **)&f.rhi, Np * nd);
    A((void **)&s->mu, N * nd);
    A((void **)&f.gf, (size_t)cell_geo_len(D) * N * nd);
    A((void **)&f.gf1, (size_t)cell_geo_len(D) * N * nd);
    A((void **)&f.pkM, (size_t)NS * NV * N * nd);
    A((void **)&f.pkR, (size_t)D * NV * N * nd);
    A((void **)&f.order, N);
    A((void **)&f.pflag, N);
    A((void **)&s->bar, 4 * sizeof(unsigned int));
    A((void **)&f.dtc, N * nd);
    double *dt0 = nullptr, *dt1 = nullptr;
    A((void **)&dt0, M->n_inst * nd);
    A((void **)&dt1, M->n_inst * nd);
    A((void **)&f.cnt, CNT_N * sizeof(int));
    A((void **)&s->tl[0], N * sizeof(int));
    A((void **)&s->tl[1], N * sizeof(int));
    A((void **)&s->nlist, Np * sizeof(int));
    A((void **)&s->clist, N * sizeof(int));
    A((void **)&s->node_mark, Np * sizeof(int));
    A((void **)&s->cell_mark, N * sizeof(int));
    A((void **)&s->totals, 8 * nd);
    A((void **)&s->ctl, sizeof(Ctl));
    A((void **)&s->d_report, sizeof(Report));
    if (r) {
        state_free(s);
        return r;
    }
    if (cudaMallocHost((void **)&s->h_cnt, CNT_N * sizeof(int)) != cudaSuccess ||
        cudaMallocHost((void **)&s->h_dt, 4 * nd) != cudaSuccess ||
        cudaMallocHost((void **)&s->h_report, sizeof(Report)) != cudaSuccess) {
        cudaGetLastError();
        state_free(s);
        return fail(LMOOD_ERR_OOM, "lmood_state_init: pinned host allocation failed");
    }
    f.m = s->m;
    f.im = s->im;
    f.mu = s->mu;
    f.dt = dt0;
    f.dtn = (unsigned long long *)dt1;
    if (dev) {  // mu > 0 checked on the device before anything else reads the inputs
        cudaMemsetAsync(f.cnt, 0, sizeof(int), st);
        k_count_nonpositive<<<256, 256, 0, st>>>(mu_cell, N, f.cnt);
        if (cudaMemcpyAsync(s->h_cnt, f.cnt, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            cudaGetLastError();
            state_free(s);
            return fail(LMOOD_ERR_CUDA, "lmood_state_init_device: checking mu");
        }
        if (s->h_cnt[0]) {
            state_free(s);
            return fail(LMOOD_ERR_ARG, "lmood_state_init_device: mu must be positive");
        }
    }
    auto H2D = [&](void *d, const void *h, size_t b) {
        if (r == LMOOD_OK &&
            cudaMemcpyAsync(d, h, b, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st) != cudaSuccess)
            r = fail(LMOOD_ERR_CUDA, "lmood_state_init: upload");
    };
    if (cudaMemcpyAsync(f.x, M->x0, D * Np * nd, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        r = fail(LMOOD_ERR_CUDA, "lmood_state_init: copy positions");
    H2D(s->mu, mu_cell, N * nd);
    H2D(f.v, v_cell, D * N * nd);
    if (F_cell) H2D(f.F, F_cell, D * D * N * nd);
    if (r == LMOOD_OK) {
        cudaMemsetAsync(s->node_mark, 0, Np * sizeof(int), st);
        cudaMemsetAsync(s->cell_mark, 0, N * sizeof(int), st);
        cudaMemsetAsync(f.vp, 0, D * Np * nd, st);
        cudaMemsetAsync(dt0, 0, M->n_inst * nd, st);
        cudaMemsetAsync(f.cnt, 0, CNT_N * sizeof(int), st);
        cudaMemsetAsync(s->ctl, 0, sizeof(Ctl), st);
        const Ops &op = *M->ops;
        Prm p0 = s->kp;
        p0.base_order = 1;
        op.init_cells(M->geo, f, p0, mat->rho0, s->m, s->im, F_cell ? 1 : 0, st);
        std::swap(s->tau, f.tau1);
        op.predict(M->geo, f, p0, nullptr, nullptr, (int)N, st);
        op.nodes(M->geo, f, nullptr, nullptr, (int)Np, 1, st);
        op.geometry(M->geo, f, st);  // the geometry record's velocity gradient, of v_p^0
        op.dt_init(f, p0, M->n_inst, 1, st);
        op.finalize(M->geo, f, p0, st);
        double *dt = const_cast<double *>(f.dt);
        f.dt = (const double *)f.dtn;
        f.dtn = (unsigned long long *)dt;
        r = sync_check(s, "lmood_state_init");
    }
    if (r) {
        state_free(s);
        return r;
    }
    s->at_init = true;
    M->states.push_back(s);
    *out = s;
    return LMOOD_OK;
}

// =======================================================================================
// step
// =======================================================================================
// The kernels of one step on stream st for the state's current buffers. Host mode stops after
// the full-mesh update (the host then drives the MOOD rounds); for graph capture the MOOD loop
// is a conditional while node whose body (two rounds, T0 -> T1 -> T0) is captured on body_st.
static void enqueue_mood_round(lmood_state s, const Fld &f, int cur, int n_in, cudaStream_t st) {
    lmood_mesh M = s->M;
    const Ops &op = *M->ops;
    const Geo &g = M->geo;
    const int N = (int)M->nc, Np = (int)M->np, NV = M->dim + 1;
    const int in = CNT_T0 + cur, out = CNT_T0 + (cur ^ 1);
    const int nb_nodes = (int)std::min<int64_t>(Np, (int64_t)NV * n_in);
    const int nb_cells = (int)std::min<int64_t>(N, (int64_t)M->max_deg * nb_nodes);
    op.round_begin(f, s->ctl, in, out, s->prm.max_mood_iters, st);
    op.mark_nodes(g, f, s->kp, s->tl[cur], f.cnt + in, n_in, s->node_mark, s->ctl, s->nlist, st);
    op.mark_cells(g, f, s->nlist, nb_nodes, s->cell_mark, s->ctl, s->clist, st);
    op.predict(g, f, s->kp, s->tl[cur], f.cnt + in, n_in, st);
    op.nodes(g, f, s->nlist, f.cnt + CNT_NODES, nb_nodes, 0, st);
    op.update(g, f, s->kp, s->clist, f.cnt + CNT_CELLS, nb_cells, s->tl[cur ^ 1], f.cnt + out, st);
}

// arguments of the persistent kernels for the state's current buffers
static PersistArgs persist_args(lmood_state s) {
    PersistArgs a{};
    a.tl0 = s->tl[0];
    a.tl1 = s->tl[1];
    a.nlist = s->nlist;
    a.clist = s->clist;
    a.node_mark = s->node_mark;
    a.cell_mark = s->cell_mark;
    a.ctl = s->ctl;
    a.report = s->d_report;
    a.bar = s->bar;
    a.max_iters = s->prm.max_mood_iters;
    a.n_inst = s->M->n_inst;
    a.max_spin = s->prm.barrier_polls > 0 ? s->prm.barrier_polls : 100000000;  // polls of ~0.1 us
    return a;
}

// zero n ints (a kernel instead of a memset node: it may sit in a conditional node's body)
__global__ static void k_zero_ints(int *p, int n) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) p[i] = 0;
}

// Enqueue one whole step on st, which is capturing into graph G: the full-mesh kernels, the
// MOOD loop as a conditional while node of G with handle h (created on G before the capture
// began; its body is captured on body_st; graph = 3: one cooperative kernel node instead),
// next dt and the step report in d_report. ev (nullptr: none) gets external event records
// around the stages for the per-stage timing; in_body: G is the body of a conditional node
// (the counters are then zeroed by a kernel rather than a memset node).
static cudaError_t capture_step(lmood_state s, cudaGraph_t G, cudaGraphConditionalHandle h, cudaStream_t st,
                                cudaEvent_t *ev, bool in_body, const char **where) {
    lmood_mesh M = s->M;
    const Ops &op = *M->ops;
    const Geo &g = M->geo;
    const Fld &f = s->f;
    const int N = (int)M->nc, Np = (int)M->np;
    auto mark = [&](int i) {
        if (ev) cudaEventRecordWithFlags(ev[i], st, cudaEventRecordExternal);
    };
    cudaError_t e = cudaSuccess;
    if (in_body)
        k_zero_ints<<<1, 32, 0, st>>>(f.cnt, CNT_N);
    else
        cudaMemsetAsync(f.cnt, 0, CNT_N * sizeof(int), st);
    op.ctl_reset(s->ctl, st);
    mark(0);
    op.moments(g, f, st);
    mark(6);
    op.predict(g, f, s->kp, nullptr, nullptr, N, st);
    mark(1);
    op.nodes(g, f, nullptr, nullptr, Np, 0, st);
    mark(2);
    op.update(g, f, s->kp, nullptr, nullptr, N, s->tl[0], f.cnt + CNT_T0, st);
    mark(3);
    *where = "capture";
    if (s->prm.graph == 3) {
        // the MOOD loop as one cooperative kernel node with grid barriers
        *where = "cooperative MOOD kernel node";
        e = cudaMemsetAsync(s->bar, 0, 4 * sizeof(unsigned int), st);
        if (e == cudaSuccess) e = op.mood_persistent(g, f, s->kp, persist_args(s), st);
    } else {
        op.loop_cond(h, f, s->ctl, st);
        cudaStreamCaptureStatus cs;
        const cudaGraphNode_t *deps = nullptr;
        size_t ndeps = 0;
        e = cudaStreamGetCaptureInfo(st, &cs, nullptr, nullptr, &deps, nullptr, &ndeps);
        cudaGraphNode_t wnode = nullptr;
        cudaGraphNodeParams cp = {};
        if (e == cudaSuccess) {
            cp.type = cudaGraphNodeTypeConditional;
            cp.conditional.handle = h;
            cp.conditional.type = cudaGraphCondTypeWhile;
            cp.conditional.size = 1;
            e = cudaGraphAddNode(&wnode, G, deps, nullptr, ndeps, &cp);
        }
        if (e == cudaSuccess)
            e = cudaStreamUpdateCaptureDependencies(st, &wnode, nullptr, 1, cudaStreamSetCaptureDependencies);
        if (e == cudaSuccess) {
            cudaGraph_t body = cp.conditional.phGraph_out[0];
            e = cudaStreamBeginCaptureToGraph(s->body_st, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                enqueue_mood_round(s, f, 0, N, s->body_st);
                enqueue_mood_round(s, f, 1, N, s->body_st);
                op.loop_cond(h, f, s->ctl, s->body_st);
                cudaGraph_t bg = nullptr;
                e = cudaStreamEndCapture(s->body_st, &bg);
            }
        }
    }
    if (e == cudaSuccess) {
        mark(4);
        op.dt_init(f, s->kp, M->n_inst, 0, st);
        op.finalize(g, f, s->kp, st);
        op.report(f, s->ctl, s->d_report, st);
        mark(5);
    }
    return e;
}

static lmood_status build_graph(lmood_state s, int par) {
    cudaStream_t st = s->cap_st;
    cudaGraph_t G = nullptr;
    LM_CUDA(cudaGraphCreate(&G, 0));
    s->graph[par] = G;
    cudaGraphConditionalHandle h{};
    if (s->prm.graph != 3) LM_CUDA(cudaGraphConditionalHandleCreate(&h, G, 0, cudaGraphCondAssignDefault));
    for (auto &e : s->gev[par]) LM_CUDA(cudaEventCreate(&e));
    cudaEvent_t *ev = s->gev[par];
    LM_CUDA(cudaStreamBeginCaptureToGraph(st, G, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    const char *where = "capture";
    cudaError_t e = capture_step(s, G, h, st, ev, false, &where);
    if (e == cudaSuccess) cudaMemcpyAsync(s->h_report, s->d_report, sizeof(Report), cudaMemcpyDeviceToHost, st);
    cudaGraph_t out = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(st, &out);
    if (e == cudaSuccess && e2 != cudaSuccess) {
        e = e2;
        where = "end of capture";
    }
    if (e == cudaSuccess) {
        where = "instantiation";
        e = cudaGraphInstantiate(&s->gexec[par], G, 0);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(LMOOD_ERR_CUDA, std::string("lmood_step: building the step graph failed (") + where +
                                        "): " + cudaGetErrorString(e));
    }
    return LMOOD_OK;
}

// chained runs: the gate of a step (run it unless an earlier step of the run failed) and
// the bookkeeping after it (accepted: count it and advance t; refused: stop the run)
__global__ static void k_run_gate(cudaGraphConditionalHandle h, const RunCtl *rc) {
    cudaGraphSetConditional(h, rc->abort == 0 ? 1u : 0u);
}

__global__ static void k_run_account(RunCtl *rc, const Report *r) {
    rc->last = *r;
    rc->ran += 1;
    if (r->err == 0 && r->n_para == 0) {
        rc->done += 1;
        rc->t += r->dt_used;
        rc->mood_pairs += (r->mood_iters + 1) / 2;
    } else {
        rc->abort = 1;
    }
}

// The chained step graph of the state's current buffer parity: k_run_gate, then an IF node
// whose body is the whole step (capture_step) followed by k_run_account.
static lmood_status build_chain_graph(lmood_state s, int par) {
    cudaStream_t st = s->cap_st;
    cudaGraph_t G = nullptr;
    LM_CUDA(cudaGraphCreate(&G, 0));
    s->cgraph[par] = G;
    cudaGraphConditionalHandle hif{};
    LM_CUDA(cudaGraphConditionalHandleCreate(&hif, G, 0, cudaGraphCondAssignDefault));
    const char *where = "gate capture";
    cudaError_t e = cudaStreamBeginCaptureToGraph(st, G, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    cudaGraphNodeParams cp = {};
    if (e == cudaSuccess) {
        k_run_gate<<<1, 1, 0, st>>>(hif, s->d_run);
        cudaStreamCaptureStatus cs;
        const cudaGraphNode_t *deps = nullptr;
        size_t ndeps = 0;
        e = cudaStreamGetCaptureInfo(st, &cs, nullptr, nullptr, &deps, nullptr, &ndeps);
        cudaGraphNode_t inode = nullptr;
        if (e == cudaSuccess) {
            cp.type = cudaGraphNodeTypeConditional;
            cp.conditional.handle = hif;
            cp.conditional.type = cudaGraphCondTypeIf;
            cp.conditional.size = 1;
            where = "IF node";
            e = cudaGraphAddNode(&inode, G, deps, nullptr, ndeps, &cp);
        }
        if (e == cudaSuccess)
            e = cudaStreamUpdateCaptureDependencies(st, &inode, nullptr, 1, cudaStreamSetCaptureDependencies);
        cudaGraph_t gout = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(st, &gout);
        if (e == cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) {
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        cudaGraphConditionalHandle hw{};
        where = "while handle in the IF body";
        e = cudaGraphConditionalHandleCreate(&hw, body, 0, cudaGraphCondAssignDefault);
        if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(st, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            e = capture_step(s, body, hw, st, nullptr, true, &where);
            if (e == cudaSuccess) k_run_account<<<1, 1, 0, st>>>(s->d_run, s->d_report);
            cudaGraph_t bout = nullptr;
            cudaError_t e2 = cudaStreamEndCapture(st, &bout);
            if (e == cudaSuccess && e2 != cudaSuccess) {
                e = e2;
                where = "end of the IF body's capture";
            }
        }
    }
    if (e == cudaSuccess) {
        where = "instantiation";
        e = cudaGraphInstantiate(&s->cexec[par], G, 0);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(LMOOD_ERR_CUDA, std::string("lmood_run: building the chained step graph failed (") + where +
                                        "): " + cudaGetErrorString(e));
    }
    return LMOOD_OK;
}

static void chain_destroy(lmood_state s) {
    for (int p = 0; p < 2; ++p) {
        if (s->cexec[p]) cudaGraphExecDestroy(s->cexec[p]);
        if (s->cgraph[p]) cudaGraphDestroy(s->cgraph[p]);
        s->cexec[p] = nullptr;
        s->cgraph[p] = nullptr;
    }
    s->chain_built = false;
}

static lmood_status ensure_chain(lmood_state s) {
    if (s->chain_built) return LMOOD_OK;
    if (!s->body_st) LM_CUDA(cudaStreamCreateWithFlags(&s->body_st, cudaStreamNonBlocking));
    if (!s->cap_st) LM_CUDA(cudaStreamCreateWithFlags(&s->cap_st, cudaStreamNonBlocking));
    if (!s->d_run) {
        lmood_status r = s->mem.alloc((void **)&s->d_run, sizeof(RunCtl));
        if (r) return r;
    }
    if (!s->h_run) LM_CUDA(cudaMallocHost((void **)&s->h_run, sizeof(RunCtl)));
    LM_CUDA(cudaStreamSynchronize(s->M->st));
    for (int k = 0; k < 2; ++k) {
        const int par = s->parity;
        lmood_status r = build_chain_graph(s, par);
        swap_state(s);
        if (r) {
            if (k == 0) swap_state(s);
            chain_destroy(s);
            return r;
        }
    }
    s->chain_built = true;
    return LMOOD_OK;
}

static lmood_status ensure_graphs(lmood_state s) {
    if (s->graphs_built) return LMOOD_OK;
    if (!s->body_st) LM_CUDA(cudaStreamCreateWithFlags(&s->body_st, cudaStreamNonBlocking));
    if (!s->cap_st) LM_CUDA(cudaStreamCreateWithFlags(&s->cap_st, cudaStreamNonBlocking));
    LM_CUDA(cudaStreamSynchronize(s->M->st));
    // graph[p] is captured with the buffers the state has when its parity is p
    for (int k = 0; k < 2; ++k) {
        const int par = s->parity;
        lmood_status r = build_graph(s, par);
        swap_state(s);
        if (r) {
            if (k == 0) swap_state(s);
            return r;
        }
    }
    s->graphs_built = true;
    return LMOOD_OK;
}

static lmood_status finish_step(lmood_state s, const Report &rep, lmood_step_info *info, int syncs) {
    lmood_step_info in{};
    in.syncs = syncs;
    in.n_troubled = rep.n_troubled;
    in.mood_iters = rep.mood_iters;
    in.n_p0 = rep.n_p0;
    in.n_parachute = rep.n_para;
    in.n_p0_eps = rep.n_eps;
    in.n_lim = rep.n_lim;
    in.dt_used = rep.dt_used;
    in.dt_next = rep.dt_next;
    in.t = s->t;
    in.step = s->step;
    if (rep.err == 2) {
        if (info) *info = in;
        return fail(LMOOD_ERR_TIMEOUT, "lmood_step: a grid barrier wait of the MOOD loop gave up; the state is unchanged");
    }
    if (rep.err) {
        if (info) *info = in;
        return fail(LMOOD_ERR_MOOD_ITERS, "lmood_step: troubled cells remain after max_mood_iters MOOD iterations");
    }
    if (in.n_parachute > 0) {
        if (info) *info = in;
        return fail(LMOOD_ERR_PARACHUTE, "lmood_step: " + std::to_string(in.n_parachute) +
                                             " first-order cells are not computable (parachute failure)");
    }
    swap_state(s);
    s->at_init = false;
    s->t += in.dt_used;
    s->step += 1;
    in.t = s->t;
    in.step = s->step;
    s->last = in;
    if (info) *info = in;
    return LMOOD_OK;
}

static lmood_status step_graph(lmood_state s, lmood_step_info *info) {
    lmood_status r = ensure_graphs(s);
    if (r) return r;
    const int par = s->parity;
    LM_CUDA(cudaGraphLaunch(s->gexec[par], s->M->st));
    if ((r = sync_check(s, "lmood_step (graph)"))) return r;
    const Report rep = *s->h_report;
    if (s->timing) {
        // event order: 0 moments 6 predict 1 nodes 2 update 3 MOOD loop 4 finalize 5
        const int from[6] = {0, 6, 1, 2, 3, 4}, to[6] = {6, 1, 2, 3, 4, 5};
        const int cls[6] = {LMOOD_K_MOMENTS, LMOOD_K_PREDICT, LMOOD_K_NODES, LMOOD_K_UPDATE, LMOOD_K_MOOD,
                            LMOOD_K_FINALIZE};
        for (int i = 0; i < 6; ++i) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, s->gev[par][from[i]], s->gev[par][to[i]]) != cudaSuccess) {
                ms = 0.f;
                cudaGetLastError();
            }
            s->kms[cls[i]] += ms;
        }
    }
    s->klaunch[LMOOD_K_MOMENTS] += 1;
    s->klaunch[LMOOD_K_PREDICT] += 1;
    s->klaunch[LMOOD_K_NODES] += 1;
    s->klaunch[LMOOD_K_UPDATE] += 1;
    if (s->prm.graph == 3)
        s->klaunch[LMOOD_K_MOOD] += 2;  // ctl reset, the cooperative MOOD kernel
    else
        s->klaunch[LMOOD_K_MOOD] += 2 + 13 * ((rep.mood_iters + 1) / 2);  // ctl reset, first condition, bodies
    s->klaunch[LMOOD_K_FINALIZE] += 3;
    return finish_step(s, rep, info, 1);
}

static lmood_status step_host(lmood_state s, lmood_step_info *info) {
    lmood_mesh M = s->M;
    const Ops &op = *M->ops;
    const Geo &g = M->geo;
    Fld &f = s->f;
    cudaStream_t st = M->st;
    const int N = (int)M->nc, Np = (int)M->np;
    LM_CUDA(cudaMemsetAsync(f.cnt, 0, CNT_N * sizeof(int), st));
    op.ctl_reset(s->ctl, st);
    timed(s, LMOOD_K_MOMENTS, 1, [&] { op.moments(g, f, st); });
    timed(s, LMOOD_K_PREDICT, 1, [&] { op.predict(g, f, s->kp, nullptr, nullptr, N, st); });
    timed(s, LMOOD_K_NODES, 1, [&] { op.nodes(g, f, nullptr, nullptr, Np, 0, st); });
    timed(s, LMOOD_K_UPDATE, 1, [&] { op.update(g, f, s->kp, nullptr, nullptr, N, s->tl[0], f.cnt + CNT_T0, st); });
    LM_CUDA(cudaMemcpyAsync(s->h_cnt, f.cnt, CNT_N * sizeof(int), cudaMemcpyDeviceToHost, st));
    lmood_status r = sync_check(s, "lmood_step");
    if (r) return r;
    int syncs = 1;
    timing_drain(s);
    int cur = 0;
    int nT = s->h_cnt[CNT_T0];
    while (nT > 0) {
        timed(s, LMOOD_K_MOOD, 6, [&] { enqueue_mood_round(s, f, cur, nT, st); });
        LM_CUDA(cudaMemcpyAsync(s->h_cnt, f.cnt, CNT_N * sizeof(int), cudaMemcpyDeviceToHost, st));
        LM_CUDA(cudaMemcpyAsync(s->h_report, s->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
        if ((r = sync_check(s, "lmood_step (MOOD)"))) return r;
        ++syncs;
        timing_drain(s);
        if (reinterpret_cast<const Ctl *>(s->h_report)->err) break;
        cur ^= 1;
        nT = s->h_cnt[CNT_T0 + cur];
    }
    timed(s, LMOOD_K_FINALIZE, 3, [&] {
        op.dt_init(f, s->kp, M->n_inst, 0, st);
        op.finalize(g, f, s->kp, st);
        op.report(f, s->ctl, s->d_report, st);
    });
    LM_CUDA(cudaMemcpyAsync(s->h_report, s->d_report, sizeof(Report), cudaMemcpyDeviceToHost, st));
    if ((r = sync_check(s, "lmood_step (finalize)"))) return r;
    timing_drain(s);
    return finish_step(s, *s->h_report, info, syncs + 1);
}

// the whole step as one cooperative launch (params.graph = 2)
static lmood_status step_persistent(lmood_state s, lmood_step_info *info) {
    lmood_mesh M = s->M;
    cudaStream_t st = M->st;
    LM_CUDA(cudaMemsetAsync(s->bar, 0, 4 * sizeof(unsigned int), st));
    const PersistArgs a = persist_args(s);
    cudaError_t e = cudaSuccess;
    timed(s, LMOOD_K_PREDICT, 1, [&] { e = M->ops->persistent(M->geo, s->f, s->kp, a, st); });
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(LMOOD_ERR_CUDA, std::string("lmood_step (persistent): launch: ") + cudaGetErrorString(e));
    }
    LM_CUDA(cudaMemcpyAsync(s->h_report, s->d_report, sizeof(Report), cudaMemcpyDeviceToHost, st));
    LM_CUDA(cudaMemcpyAsync(s->h_cnt, s->bar + 2, sizeof(unsigned int), cudaMemcpyDeviceToHost, st));
    lmood_status r = sync_check(s, "lmood_step (persistent)");
    if (r) return r;
    timing_drain(s);
    if (s->h_cnt[0] != 0)
        return fail(LMOOD_ERR_TIMEOUT, "lmood_step (persistent): a grid barrier wait gave up; the state is unchanged");
    return finish_step(s, *s->h_report, info, 1);
}

extern "C" lmood_status lmood_step(lmood_state s, lmood_step_info *info) {
    if (!s) return fail(LMOOD_ERR_ARG, "lmood_step: NULL state");
    if (s->broken) return fail(LMOOD_ERR_STATE, "lmood_step: state unusable after an earlier CUDA error");
    if (s->prm.graph == 2) return step_persistent(s, info);
    return s->prm.graph ? step_graph(s, info) : step_host(s, info);
}

// nsteps chained step graphs launched back to back, one synchronisation at the end: each
// step runs only if every earlier step of the run was accepted (k_run_gate), and the state
// then holds the last accepted step, exactly as after that many lmood_step calls.
static lmood_status run_chained(lmood_state s, int64_t nsteps, lmood_step_info *last) {
    lmood_status r = ensure_chain(s);
    if (r) return r;
    cudaStream_t st = s->M->st;
    RunCtl init{};
    init.t = s->t;
    *s->h_run = init;
    LM_CUDA(cudaMemcpyAsync(s->d_run, s->h_run, sizeof(RunCtl), cudaMemcpyHostToDevice, st));
    const int par0 = s->parity;
    for (int64_t i = 0; i < nsteps; ++i) LM_CUDA(cudaGraphLaunch(s->cexec[(par0 + i) & 1], st));
    LM_CUDA(cudaMemcpyAsync(s->h_run, s->d_run, sizeof(RunCtl), cudaMemcpyDeviceToHost, st));
    if ((r = sync_check(s, "lmood_run (chained steps)"))) return r;
    const RunCtl rc = *s->h_run;
    s->klaunch[LMOOD_K_FINALIZE] += nsteps + 4 * (int64_t)rc.ran;  // gates; dt_init, finalize, report, account
    s->klaunch[LMOOD_K_MOMENTS] += rc.ran;
    s->klaunch[LMOOD_K_PREDICT] += rc.ran;
    s->klaunch[LMOOD_K_NODES] += rc.ran;
    s->klaunch[LMOOD_K_UPDATE] += rc.ran;
    s->klaunch[LMOOD_K_MOOD] += 3 * (int64_t)rc.ran + 13 * (int64_t)rc.mood_pairs;
    // the accepted steps, as lmood_step would have left the state after each
    for (int i = 0; i < rc.done; ++i) swap_state(s);
    if (rc.done > 0) s->at_init = false;
    s->step += rc.done;
    s->t = rc.t;
    if (rc.ran == rc.done) {
        // every step was accepted: the report of the last one
        lmood_step_info in{};
        const Report &rep = rc.last;
        in.n_troubled = rep.n_troubled;
        in.mood_iters = rep.mood_iters;
        in.n_p0 = rep.n_p0;
        in.n_parachute = rep.n_para;
        in.n_p0_eps = rep.n_eps;
        in.n_lim = rep.n_lim;
        in.dt_used = rep.dt_used;
        in.dt_next = rep.dt_next;
        in.t = s->t;
        in.step = s->step;
        in.syncs = 1;
        s->last = in;
        if (last) *last = in;
        return LMOOD_OK;
    }
    // the failing step (refused by finish_step's rules; the state holds the steps before it)
    return finish_step(s, rc.last, last, 1);
}

extern "C" lmood_status lmood_run(lmood_state s, int64_t nsteps, lmood_step_info *last) {
    if (!s || nsteps < 0) return fail(LMOOD_ERR_ARG, "lmood_run: bad argument");
    if (s->broken) return fail(LMOOD_ERR_STATE, "lmood_run: state unusable after an earlier CUDA error");
    if (nsteps >= 2 && s->prm.graph == 1 && !s->timing && !s->chain_unsupported) {
        lmood_status r = run_chained(s, nsteps, last);
        if (r != LMOOD_ERR_CUDA || s->chain_built || s->broken) return r;
        // the chained graph could not be built on this device / driver: step one at a time
        s->chain_unsupported = true;
        s->chain_err = lmood_last_error();
    }
    int syncs = 0;
    for (int64_t i = 0; i < nsteps; ++i) {
        lmood_status r = lmood_step(s, last);
        syncs += s->last.syncs;
        if (r) return r;
    }
    if (last) {
        if (nsteps == 0) *last = s->last;
        last->syncs = syncs;
    }
    return LMOOD_OK;
}

// =======================================================================================
// fields
// =======================================================================================
__global__ static void k_u8_to_f64(const unsigned char *a, double *b, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = a[i];
}

// device source of a readable field (ORDER is converted to doubles in scratch first)
static lmood_status get_source(lmood_state s, int field, const void **src, size_t *bytes) {
    lmood_mesh M = s->M;
    const int D = M->dim, NV = D + 1, NS = D * (D + 1) / 2;
    const size_t N = M->nc, Np = M->np, nd = sizeof(double);
    const Fld &f = s->f;
    switch (field) {
    case LMOOD_FIELD_X: *src = f.x; *bytes = D * Np * nd; break;
    case LMOOD_FIELD_VP: *src = f.vp; *bytes = D * Np * nd; break;
    case LMOOD_FIELD_VSTAR: *src = f.vs; *bytes = D * Np * nd; break;
    case LMOOD_FIELD_V: *src = f.v; *bytes = D * N * nd; break;
    case LMOOD_FIELD_E: *src = f.e; *bytes = N * nd; break;
    case LMOOD_FIELD_F: *src = f.F; *bytes = D * D * N * nd; break;
    case LMOOD_FIELD_TAU: *src = s->tau; *bytes = N * nd; break;
    case LMOOD_FIELD_MASS: *src = s->m; *bytes = N * nd; break;
    case LMOOD_FIELD_PKM: *src = f.pkM; *bytes = NS * NV * N * nd; break;
    case LMOOD_FIELD_PKR: *src = f.pkR; *bytes = D * NV * N * nd; break;
    case LMOOD_FIELD_DT: *src = f.dt; *bytes = M->n_inst * nd; break;
    case LMOOD_FIELD_ORDER: {
        double *tmp = (double *)f.dtc;  // the dt candidates are rebuilt every step
        k_u8_to_f64<<<(unsigned)((N + 255) / 256), 256, 0, M->st>>>(f.order, tmp, (int)N);
        *src = tmp;
        *bytes = N * nd;
        break;
    }
    default: return fail(LMOOD_ERR_ARG, "lmood_get: unknown field id");
    }
    return LMOOD_OK;
}

// device destination of a settable field
static lmood_status set_target(lmood_state s, int field, void **dst, size_t *bytes) {
    lmood_mesh M = s->M;
    const int D = M->dim;
    const size_t N = M->nc, Np = M->np, nd = sizeof(double);
    Fld &f = s->f;
    switch (field) {
    case LMOOD_FIELD_X: *dst = f.x; *bytes = D * Np * nd; break;
    case LMOOD_FIELD_VP: *dst = f.vp; *bytes = D * Np * nd; break;
    case LMOOD_FIELD_V: *dst = f.v; *bytes = D * N * nd; break;
    case LMOOD_FIELD_E: *dst = f.e; *bytes = N * nd; break;
    case LMOOD_FIELD_F: *dst = f.F; *bytes = D * D * N * nd; break;
    case LMOOD_FIELD_DT: *dst = const_cast<double *>(f.dt); *bytes = M->n_inst * nd; break;
    default: return fail(LMOOD_ERR_ARG, "lmood_set: unknown or read-only field id");
    }
    return LMOOD_OK;
}

extern "C" lmood_status lmood_get_fields(lmood_state s, int n, const int *fields, void *const *dst, int is_device) {
    if (!s || n < 0 || (n > 0 && (!fields || !dst))) return fail(LMOOD_ERR_ARG, "lmood_get_fields: bad argument");
    if (!s->M) return fail(LMOOD_ERR_STATE, "lmood_get_fields: the state's mesh was destroyed");
    for (int i = 0; i < n; ++i) {
        if (!dst[i]) return fail(LMOOD_ERR_ARG, "lmood_get_fields: NULL destination");
        if (fields[i] < 0 || fields[i] > LMOOD_FIELD_DT) return fail(LMOOD_ERR_ARG, "lmood_get_fields: unknown field id");
        for (int j = 0; j < i; ++j)  // ORDER shares its scratch: at most once per call
            if (fields[i] == LMOOD_FIELD_ORDER && fields[j] == LMOOD_FIELD_ORDER)
                return fail(LMOOD_ERR_ARG, "lmood_get_fields: ORDER requested twice");
    }
    cudaStream_t st = s->M->st;
    for (int i = 0; i < n; ++i) {
        const void *src = nullptr;
        size_t bytes = 0;
        lmood_status r = get_source(s, fields[i], &src, &bytes);
        if (r) return r;
        LM_CUDA(cudaMemcpyAsync(dst[i], src, bytes, is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    }
    if (!is_device) return sync_check(s, "lmood_get_fields");
    return LMOOD_OK;
}

extern "C" lmood_status lmood_set_fields(lmood_state s, int n, const int *fields, const void *const *src, int is_device) {
    if (!s || n < 0 || (n > 0 && (!fields || !src))) return fail(LMOOD_ERR_ARG, "lmood_set_fields: bad argument");
    if (!s->M) return fail(LMOOD_ERR_STATE, "lmood_set_fields: the state's mesh was destroyed");
    for (int i = 0; i < n; ++i) {  // validate everything before the first copy
        void *dst = nullptr;
        size_t bytes = 0;
        if (!src[i]) return fail(LMOOD_ERR_ARG, "lmood_set_fields: NULL source");
        lmood_status r = set_target(s, fields[i], &dst, &bytes);
        if (r) return r;
    }
    lmood_mesh M = s->M;
    cudaStream_t st = M->st;
    auto is_geo = [&](int i) {
        return fields[i] == LMOOD_FIELD_X || fields[i] == LMOOD_FIELD_VP || fields[i] == LMOOD_FIELD_F;
    };
    int n_geo = 0, n_eps = 0;  // (the stiffened gas's impedance depends on eps = e - |v|^2 / 2 too)
    for (int i = 0; i < n; ++i) {
        n_geo += is_geo(i);
        n_eps += s->mat.eos != 0 && (fields[i] == LMOOD_FIELD_V || fields[i] == LMOOD_FIELD_E);
    }
    // derived cell geometry (with the velocity gradient of v_p), density and impedance from the
    // new x, v_p and F; the refresh reads nothing else for the volumetric law of Eq.
    // EOS_neoHook, so it runs on a side stream while the other fields are copied (the stiffened
    // gas's impedance also needs v and e)
    const bool side = n_geo > 0 && n_geo < n && s->mat.eos == 0;
    auto refresh = [&](cudaStream_t rs) {
        Fld &f = s->f;
        std::swap(s->tau, f.tau1);
        M->ops->refresh(M->geo, f, s->kp, rs);
        std::swap(s->tau, f.tau1);
    };
    if (side && !s->aux_st) {
        LM_CUDA(cudaStreamCreateWithFlags(&s->aux_st, cudaStreamNonBlocking));
        for (auto &e : s->set_ev) LM_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    for (int pass = 0; pass < 2; ++pass) {  // X, v_p and F first
        for (int i = 0; i < n; ++i) {
            if (is_geo(i) != (pass == 0)) continue;
            void *dst = nullptr;
            size_t bytes = 0;
            set_target(s, fields[i], &dst, &bytes);
            LM_CUDA(cudaMemcpyAsync(dst, src[i], bytes, is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
            if (fields[i] != LMOOD_FIELD_DT) s->at_init = false;
        }
        if (pass == 0 && side) {
            LM_CUDA(cudaEventRecord(s->set_ev[0], st));
            LM_CUDA(cudaStreamWaitEvent(s->aux_st, s->set_ev[0], 0));
            refresh(s->aux_st);
            LM_CUDA(cudaEventRecord(s->set_ev[1], s->aux_st));
        }
    }
    if (side) LM_CUDA(cudaStreamWaitEvent(st, s->set_ev[1], 0));
    else if (n_geo > 0 || n_eps > 0) refresh(st);
    if (!is_device) return sync_check(s, "lmood_set_fields");
    return LMOOD_OK;
}

extern "C" lmood_status lmood_get(lmood_state s, int field, void *dst, int is_device) {
    if (!s || !dst) return fail(LMOOD_ERR_ARG, "lmood_get: NULL argument");
    return lmood_get_fields(s, 1, &field, &dst, is_device);
}

extern "C" lmood_status lmood_set(lmood_state s, int field, const void *src, int is_device) {
    if (!s || !src) return fail(LMOOD_ERR_ARG, "lmood_set: NULL argument");
    return lmood_set_fields(s, 1, &field, &src, is_device);
}

extern "C" lmood_status lmood_totals(lmood_state s, double *out5) {
    if (!s || !out5) return fail(LMOOD_ERR_ARG, "lmood_totals: NULL argument");
    if (!s->M) return fail(LMOOD_ERR_STATE, "lmood_totals: the state's mesh was destroyed");
    cudaStream_t st = s->M->st;
    LM_CUDA(cudaMemsetAsync(s->totals, 0, 5 * sizeof(double), st));
    s->M->ops->totals(s->M->geo, s->f, s->totals, st);
    LM_CUDA(cudaMemcpyAsync(out5, s->totals, 5 * sizeof(double), cudaMemcpyDeviceToHost, st));
    return sync_check(s, "lmood_totals");
}

// the state's captured step graphs (re-captured at the next step)
static void graphs_destroy(lmood_state s) {
    chain_destroy(s);
    for (int p = 0; p < 2; ++p) {
        if (s->gexec[p]) cudaGraphExecDestroy(s->gexec[p]);
        if (s->graph[p]) cudaGraphDestroy(s->graph[p]);
        s->gexec[p] = nullptr;
        s->graph[p] = nullptr;
        for (cudaEvent_t &e : s->gev[p]) {
            if (e) cudaEventDestroy(e);
            e = nullptr;
        }
    }
    s->graphs_built = false;
}

void lmood::graphs_reset(lmood_state_s *s) { graphs_destroy(s); }

extern "C" lmood_status lmood_autotune(lmood_state s, int reps, double *ms12, int32_t *chosen4) {
    if (!s) return fail(LMOOD_ERR_ARG, "lmood_autotune: NULL state");
    if (s->broken) return fail(LMOOD_ERR_STATE, "lmood_autotune: state unusable after an earlier CUDA error");
    if (reps <= 0) reps = 5;
    lmood_mesh M = s->M;
    const Ops &op = *M->ops;
    cudaStream_t st = M->st;
    Fld &f = s->f;
    const int N = (int)M->nc, Np = (int)M->np;
    // the kernels run on the state's current fields with their current orders and no
    // detection: they only rewrite scratch (moments, packets, v*, candidate state)
    Prm kt = s->kp;
    kt.base_order = 0;
    kt.mood = 0;
    cudaEvent_t e0, e1;
    LM_CUDA(cudaEventCreate(&e0));
    LM_CUDA(cudaEventCreate(&e1));
    const int cand[4][3] = {{128, 256, 512}, {64, 128, 256}, {128, 256, 512}, {64, 128, 256}};  // moments, predict, nodes, update
    int *slot[4] = {&M->geo.blk.moments, &M->geo.blk.predict, &M->geo.blk.nodes, &M->geo.blk.update};
    double times[4][3] = {};
    cudaError_t err = cudaSuccess;
    for (int k = 0; k < 4 && err == cudaSuccess; ++k) {
        int best = *slot[k];
        double best_ms = 1e300;
        for (int v = 0; v < 3 && err == cudaSuccess; ++v) {
            *slot[k] = cand[k][v];
            const Geo &g = M->geo;
            auto launch = [&] {
                switch (k) {
                case 0: op.moments(g, f, st); break;
                case 1: op.predict(g, f, kt, nullptr, nullptr, N, st); break;
                case 2: op.nodes(g, f, nullptr, nullptr, Np, 0, st); break;
                default: op.update(g, f, kt, nullptr, nullptr, N, s->tl[0], f.cnt + CNT_T0, st); break;
                }
            };
            launch();  // warm
            cudaEventRecord(e0, st);
            for (int r = 0; r < reps; ++r) launch();
            cudaEventRecord(e1, st);
            err = cudaEventSynchronize(e1);
            if (err == cudaSuccess) err = cudaGetLastError();
            float ms = 0.f;
            if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
            times[k][v] = ms / reps;
            if (times[k][v] < best_ms) {
                best_ms = times[k][v];
                best = cand[k][v];
            }
        }
        *slot[k] = best;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess) {
        s->broken = true;
        return fail(LMOOD_ERR_CUDA, std::string("lmood_autotune: ") + cudaGetErrorString(err));
    }
    graphs_destroy(s);  // re-captured with the chosen launch shapes at the next step
    if (ms12)
        for (int k = 0; k < 4; ++k)
            for (int v = 0; v < 3; ++v) ms12[k * 3 + v] = times[k][v];
    if (chosen4)
        for (int k = 0; k < 4; ++k) chosen4[k] = *slot[k];
    return LMOOD_OK;
}

// ---------------------------------------------------------------------------------------
// schedule autotuning: the node order of the whole-mesh node kernels and the step form
// ---------------------------------------------------------------------------------------
// the nodes of each window of W consecutive ones in order of their cell count (stable; W <= 0:
// the nodes in their own order)
static void node_order(const std::vector<int> &off, int64_t W, std::vector<int> &perm) {
    const int64_t Np = (int64_t)off.size() - 1;
    perm.resize(Np);
    if (W <= 0) {
        for (int64_t p = 0; p < Np; ++p) perm[p] = (int)p;
        return;
    }
    int max_deg = 0;
    for (int64_t p = 0; p < Np; ++p) max_deg = std::max(max_deg, off[p + 1] - off[p]);
    std::vector<int64_t> first(max_deg + 2);
    for (int64_t w0 = 0; w0 < Np; w0 += W) {
        const int64_t w1 = std::min(Np, w0 + W);
        std::fill(first.begin(), first.end(), 0);
        for (int64_t p = w0; p < w1; ++p) first[off[p + 1] - off[p] + 1]++;
        first[0] = w0;
        for (int d2 = 0; d2 <= max_deg; ++d2) first[d2 + 1] += first[d2];
        for (int64_t p = w0; p < w1; ++p) perm[first[off[p + 1] - off[p]]++] = (int)p;
    }
}

// the dynamic state of s (the fields a step reads and writes, and the host counters), copied
// aside on the device so that trial steps can be undone exactly
struct StateCopy {
    std::vector<std::pair<void *, size_t>> parts;  // (device copy, bytes) in the order of fields()
    double t = 0.0;
    int64_t step = 0;
    bool at_init = false;
    lmood_step_info last{};
    static std::vector<std::pair<void *, size_t>> fields(lmood_state s) {
        lmood_mesh M = s->M;
        const size_t D = M->dim, N = M->nc, Np = M->np, nd = sizeof(double);
        Fld &f = s->f;
        return {{f.x, D * Np * nd}, {f.vp, D * Np * nd}, {f.v, D * N * nd}, {f.e, N * nd}, {f.F, D * D * N * nd},
                {f.xc, D * N * nd}, {f.rho, N * nd}, {f.z, N * nd}, {s->tau, N * nd}, {f.order, N},
                {f.gf, (size_t)cell_geo_len((int)D) * N * nd},
                {const_cast<double *>(f.dt), (size_t)M->n_inst * nd}};
    }
    lmood_status save(lmood_state s) {
        for (auto &pb : fields(s)) {
            void *d = nullptr;
            if (cudaMalloc(&d, pb.second) != cudaSuccess) {
                cudaGetLastError();
                release();
                return fail(LMOOD_ERR_OOM, "lmood_autotune_schedule: no device memory for the state copy");
            }
            parts.push_back({d, pb.second});
            LM_CUDA(cudaMemcpyAsync(d, pb.first, pb.second, cudaMemcpyDeviceToDevice, s->M->st));
        }
        t = s->t;
        step = s->step;
        at_init = s->at_init;
        last = s->last;
        return LMOOD_OK;
    }
    // into the state's current buffers (whichever parity the trial steps left)
    lmood_status restore(lmood_state s) {
        auto cur = fields(s);
        for (size_t i = 0; i < cur.size(); ++i)
            LM_CUDA(cudaMemcpyAsync(cur[i].first, parts[i].first, parts[i].second, cudaMemcpyDeviceToDevice, s->M->st));
        s->t = t;
        s->step = step;
        s->at_init = at_init;
        s->last = last;
        return LMOOD_OK;
    }
    void release() {
        for (auto &pb : parts) cudaFree(pb.first);
        parts.clear();
    }
};

extern "C" lmood_status lmood_autotune_schedule(lmood_state s, int reps, double *ms_window4, int32_t *window,
                                                double *ms_form2, int32_t *form) {
    if (!s) return fail(LMOOD_ERR_ARG, "lmood_autotune_schedule: NULL state");
    if (s->broken) return fail(LMOOD_ERR_STATE, "lmood_autotune_schedule: state unusable after an earlier CUDA error");
    if (s->timing) return fail(LMOOD_ERR_ARG, "lmood_autotune_schedule: switch timing off first");
    if (reps <= 0) reps = 5;
    lmood_mesh M = s->M;
    const Ops &op = *M->ops;
    cudaStream_t st = M->st;
    Fld &f = s->f;
    const int Np = (int)M->np;
    cudaEvent_t e0, e1;
    LM_CUDA(cudaEventCreate(&e0));
    LM_CUDA(cudaEventCreate(&e1));
    lmood_status r = LMOOD_OK;
    // 1. node order: the moments and the nodal solve over the whole mesh, per window size
    const int cand[4] = {32, 256, 2048, 0};
    double tw[4] = {};
    std::vector<int> off(Np + 1), perm;
    int *d_perm = const_cast<int *>(M->geo.node_perm);
    cudaError_t err = cudaMemcpyAsync(off.data(), M->geo.n2c_off, (Np + 1) * sizeof(int), cudaMemcpyDeviceToHost, st);
    if (err == cudaSuccess) err = cudaStreamSynchronize(st);
    int best = 1;
    for (int v = 0; v < 4 && err == cudaSuccess; ++v) {
        node_order(off, cand[v], perm);
        err = cudaMemcpyAsync(d_perm, perm.data(), Np * sizeof(int), cudaMemcpyHostToDevice, st);
        if (err != cudaSuccess) break;
        auto launch = [&] {
            op.moments(M->geo, f, st);
            op.nodes(M->geo, f, nullptr, nullptr, Np, 0, st);
        };
        launch();  // warm
        cudaEventRecord(e0, st);
        for (int k = 0; k < reps; ++k) launch();
        cudaEventRecord(e1, st);
        err = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
        tw[v] = ms / reps;
        if (tw[v] < tw[best]) best = v;
    }
    if (err == cudaSuccess) {
        node_order(off, cand[best], perm);
        err = cudaMemcpyAsync(d_perm, perm.data(), Np * sizeof(int), cudaMemcpyHostToDevice, st);
        if (err == cudaSuccess) err = cudaStreamSynchronize(st);
    }
    if (err != cudaSuccess) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        s->broken = true;
        return fail(LMOOD_ERR_CUDA, std::string("lmood_autotune_schedule: ") + cudaGetErrorString(err));
    }
    if (ms_window4)
        for (int v = 0; v < 4; ++v) ms_window4[v] = tw[v];
    if (window) *window = cand[best];
    // 2. step form: reps steps (lmood_step, host synchronisation included) from the state as it
    // is, once per form, the state restored after each; only between the captured form (1) and
    // the persistent one (2), and only where the persistent form applies (neo-Hookean material)
    double tf[2] = {-1.0, -1.0};
    int chosen = s->prm.graph;
    const bool both = (s->prm.graph == 1 || s->prm.graph == 2) && s->mat.shear_a == -1.0 && s->mat.eos == 0;
    if (both) {
        StateCopy keep;
        r = keep.save(s);
        const int g0 = s->prm.graph;
        for (int v = 0; v < 2 && r == LMOOD_OK; ++v) {
            s->prm.graph = v + 1;
            r = lmood_step(s, nullptr);  // warm (graphs captured, lists sized)
            if (r == LMOOD_OK) r = keep.restore(s);
            if (r == LMOOD_OK && cudaStreamSynchronize(st) != cudaSuccess) r = sync_check(s, "lmood_autotune_schedule");
            const auto t0 = std::chrono::steady_clock::now();
            for (int k = 0; k < reps && r == LMOOD_OK; ++k) r = lmood_step(s, nullptr);
            const auto t1 = std::chrono::steady_clock::now();
            tf[v] = std::chrono::duration<double, std::milli>(t1 - t0).count() / reps;
            if (r == LMOOD_OK) r = keep.restore(s);
        }
        if (r == LMOOD_OK) r = sync_check(s, "lmood_autotune_schedule (restore)");
        keep.release();
        s->prm.graph = g0;
        if (r == LMOOD_OK) {
            chosen = tf[1] < tf[0] ? 2 : 1;
            s->prm.graph = chosen;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (r) return r;
    if (ms_form2) {
        ms_form2[0] = tf[0];
        ms_form2[1] = tf[1];
    }
    if (form) *form = both ? chosen : -1;
    return LMOOD_OK;
}

extern "C" lmood_status lmood_timing(lmood_state s, int enable) {
    if (!s) return fail(LMOOD_ERR_ARG, "lmood_timing: NULL state");
    if (!s->M) return fail(LMOOD_ERR_STATE, "lmood_timing: the state's mesh was destroyed");
    if (enable && s->ev.empty()) {
        s->ev.resize(2 * kMaxPending);
        for (auto &e : s->ev) LM_CUDA(cudaEventCreate(&e));
    }
    LM_CUDA(cudaStreamSynchronize(s->M->st));
    timing_drain(s);
    if (enable) {
        for (int i = 0; i < LMOOD_NK; ++i) {
            s->kms[i] = 0;
            s->klaunch[i] = 0;
        }
    }
    s->timing = enable != 0;
    return LMOOD_OK;
}

extern "C" lmood_status lmood_timing_read(lmood_state s, double *ms, int64_t *launches) {
    if (!s || !ms || !launches) return fail(LMOOD_ERR_ARG, "lmood_timing_read: NULL argument");
    if (!s->M) return fail(LMOOD_ERR_STATE, "lmood_timing_read: the state's mesh was destroyed");
    for (int i = 0; i < LMOOD_NK; ++i) {
        ms[i] = s->kms[i];
        launches[i] = s->klaunch[i];
    }
    return LMOOD_OK;
}

extern "C" const char *lmood_last_error(void) { return g_err.c_str(); }
