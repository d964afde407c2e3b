// lmood_internal.h -- host-side objects behind the opaque handles of include/lmood.h (mesh,
// state) and the helpers the library's translation units share. Not part of the C ABI.
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "lmood.h"
#include "lmood_ops.h"

namespace lmood {

// control block of a device-chained run: the steps that ran and were accepted, the time
// after the last accepted one (accumulated in the order lmood_step does), the MOOD loop's
// body launches (for the launch counts) and the report of the last step that ran
struct RunCtl {
    int abort, ran, done, mood_pairs;
    double t;
    Report last;
};

// sets the calling thread's last error message (read back with lmood_last_error) and returns st
lmood_status fail(lmood_status st, const std::string &msg);

#define LM_CUDA(call)                                                                          \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess) return ::lmood::fail(LMOOD_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// device allocations owned by one object, freed together
struct DevAllocs {
    std::vector<void *> ptrs;
    lmood_status alloc(void **p, size_t bytes) {
        *p = nullptr;
        if (bytes == 0) bytes = 16;
        cudaError_t e = cudaMalloc(p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            // out of device memory, or no usable device / driver at all
            return fail(e == cudaErrorMemoryAllocation ? LMOOD_ERR_OOM : LMOOD_ERR_CUDA,
                        std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
        }
        ptrs.push_back(*p);
        return LMOOD_OK;
    }
    void release() {
        for (void *p : ptrs) cudaFree(p);
        ptrs.clear();
    }
};

}  // namespace lmood

struct lmood_mesh_s {
    int dim = 0, n_inst = 1;
    int64_t np = 0, nc = 0, st_nnz = 0, nb = 0;
    int max_deg = 0;
    cudaStream_t st = nullptr;
    const lmood::Ops *ops = nullptr;
    lmood::Geo geo{};
    double *x0 = nullptr;
    // host copies for re-deriving the node conditions when the face tags change
    std::vector<double> h_x0;     // [dim][np]
    std::vector<int> h_bf;        // [dim][nb], oriented outward
    std::vector<int> h_btag;      // [nb]
    unsigned char *d_ndof = nullptr, *d_btag = nullptr;
    double *d_bct = nullptr, *d_bfval = nullptr, *d_contact = nullptr;
    bool has_ext = false;         // some face has a traction / pressure / velocity / contact tag
    uint64_t bc_version = 0;      // counts the changes of boundary values, tags and contact walls
    std::vector<lmood_state_s *> states;  // the live states on this mesh (orphaned when it goes)
    lmood::DevAllocs mem;
};

struct lmood_tape_s;
struct lmood_state_s {
    lmood_mesh M = nullptr;          // NULL once the mesh was destroyed first: unusable but destroyable
    std::vector<lmood_tape_s *> tapes;  // the live tapes of this state (orphaned when it goes)
    lmood_params prm{};
    lmood_material mat{};
    lmood::Prm kp{};
    lmood::Fld f{};
    double *tau = nullptr, *m = nullptr, *im = nullptr, *mu = nullptr;
    int *tl[2] = {nullptr, nullptr}, *nlist = nullptr, *clist = nullptr, *node_mark = nullptr, *cell_mark = nullptr;
    double *totals = nullptr;
    lmood::Ctl *ctl = nullptr;   // device MOOD control block
    lmood::Report *d_report = nullptr;
    lmood::Report *h_report = nullptr;  // pinned
    // graph-captured steps: one executable graph per buffer parity (the state swaps pointers)
    int parity = 0;
    bool graphs_built = false;
    cudaGraph_t graph[2] = {nullptr, nullptr};
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    cudaEvent_t gev[2][7] = {};
    cudaStream_t cap_st = nullptr;   // private streams for capturing (the mesh's stream may be the
    cudaStream_t body_st = nullptr;  // legacy default stream, which cannot be captured)
    // device-chained runs (lmood_run): per buffer parity a graph whose step sits in an IF node
    // gated by the run's abort word, so that the steps of a run need no host synchronisation
    bool chain_built = false, chain_unsupported = false;
    std::string chain_err;                       // why the chained form could not be built
    cudaGraph_t cgraph[2] = {nullptr, nullptr};
    cudaGraphExec_t cexec[2] = {nullptr, nullptr};
    lmood::RunCtl *d_run = nullptr;              // the run's control block (device)
    lmood::RunCtl *h_run = nullptr;              //   and its pinned mirror
    unsigned int *bar = nullptr;  // persistent step: grid barrier state (device, 4 words)
    cudaStream_t aux_st = nullptr;   // lmood_set_fields: the geometry refresh beside the copies
    cudaEvent_t set_ev[2] = {};      //   (X and F copied; refresh done)
    int *h_cnt = nullptr;      // pinned mirror of the device counters
    double *h_dt = nullptr;    // pinned: dt used, dt next (instance 0)
    double t = 0.0;
    int64_t step = 0;
    int stamp = 0;
    bool broken = false;
    // true from lmood_state_init until the first step or lmood_set: v_p is then the initial
    // nodal solve of (v, F, mu), which a tape recorded from here differentiates through
    bool at_init = false;
    lmood_step_info last{};
    // kernel timing (CUDA events around launches, drained at the step's sync points)
    bool timing = false;
    std::vector<cudaEvent_t> ev;            // pool of 2 * kMaxPending events
    std::vector<int> pend_cls;              // class of each pending pair
    double kms[LMOOD_NK] = {};
    int64_t klaunch[LMOOD_NK] = {};
    lmood::DevAllocs mem;
};

namespace lmood {

// exchanges the t^n and t^{n+1} buffers of the state (and dt / dt next), toggling its parity
void swap_state(lmood_state s);
// synchronises the mesh stream; a CUDA error marks the state unusable
lmood_status sync_check(lmood_state s, const char *where);

}  // namespace lmood

namespace lmood {
// the state is going: its remaining tapes become orphans (destroyable, nothing else)
void tapes_orphan(lmood_state_s *s);
// drop the state's captured step graphs (they hold its field pointers; re-captured at the next step)
void graphs_reset(lmood_state_s *s);
}  // namespace lmood
