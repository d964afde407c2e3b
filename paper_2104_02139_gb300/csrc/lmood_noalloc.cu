// lmood_noalloc.cu -- lmood_totals_noalloc: the conserved totals (mass, momentum, total
// energy) of caller-owned cell arrays, computed without allocating any device memory.
//
// Who needs it: host applications that own every device allocation themselves and forbid
// libraries from allocating after start-up -- for example coupled multi-physics codes that
// carve all GPU memory out of one pool at initialisation, or real-time loops in which a
// cudaMalloc (which may synchronise the device and can fail under fragmentation) is not
// allowed. lmood_totals needs a small device buffer that the library allocates with the
// state; this variant keeps its scratch in a fixed file-scope device array instead.
//
// Scratch: g_totals_scratch holds one row of partial sums per block, 4,096 rows of 8 doubles
// (256 KiB), so at most 4,096 blocks x 4,096 cells = 16,777,216 cells per call. Every GPU
// that loads this library holds the array until the process exits. All calls share it and it
// keeps the last call's partial sums; each call overwrites exactly the rows it reads, so
// nothing needs clearing, but calls whose kernels overlap on the GPU (different streams, or
// other host threads) race on the array and must be ordered by the caller.
#include <cuda.h>

#include <mutex>
#include <string>

#include "lmood.h"

void lmood_internal_set_error(const char *msg);  // lmood_api.cu

// the scratch array (see above); host code uses its address from cudaGetSymbolAddress only
static __device__ __align__(256) double g_totals_scratch[4096 * 8];

namespace {

constexpr int kBlock = 256;
constexpr int kPerThread = 16;
constexpr int kCellsPerBlock = kBlock * kPerThread;  // 4,096
constexpr int kMaxBlocks = 4096;
constexpr int64_t kMaxCells = (int64_t)kMaxBlocks * kCellsPerBlock;
constexpr int kRow = 8;  // mass, mom x, y, z, energy, 3 spare

static_assert(sizeof(g_totals_scratch) == sizeof(double) * kMaxBlocks * kRow, "scratch size");

// Device address of g_totals_scratch per device, looked up (with that device current) on the
// first call made on it; host code must not use the symbol itself as an address. The address
// belongs to the device's current CUDA context: after a cudaDeviceReset the runtime creates a
// new context and loads the module again, so the cache also keeps the id of the context the
// address was taken in and looks the address up again when that id changes.
constexpr int kMaxDevices = 64;
double *g_scratch_ptr[kMaxDevices] = {nullptr};
unsigned long long g_scratch_ctx[kMaxDevices] = {0};
std::mutex g_scratch_mu;

// the driver's cuCtxGetCurrent / cuCtxGetId through the runtime's entry-point query (no link
// against the driver library, which a machine without a GPU does not have)
typedef CUresult (*PfnCtxGetCurrent)(CUcontext *);
typedef CUresult (*PfnCtxGetId)(CUcontext, unsigned long long *);

// id of the calling thread's current context (0 when it cannot be determined: the cache then
// never matches and the address is looked up on every call)
unsigned long long current_context_id() {
    static PfnCtxGetCurrent get_current = nullptr;
    static PfnCtxGetId get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = (PfnCtxGetCurrent)f;
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = (PfnCtxGetId)f;
        cudaGetLastError();
    });
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
        return 0;
    return id;
}

lmood_status fail(lmood_status s, const std::string &m) {
    lmood_internal_set_error(m.c_str());  // read back with lmood_last_error()
    return s;
}

// Fixed-order block reduction of 5 values (shared-memory tree), result in thread 0.
__device__ void block_sum5(double (&q)[5], double (*sh)[kBlock]) {
    for (int i = 0; i < 5; ++i) sh[i][threadIdx.x] = q[i];
    __syncthreads();
    for (int w = kBlock / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int i = 0; i < 5; ++i) sh[i][threadIdx.x] += sh[i][threadIdx.x + w];
        __syncthreads();
    }
    for (int i = 0; i < 5; ++i) q[i] = sh[i][0];
}

__global__ void __launch_bounds__(kBlock) k_partials(int dim, int64_t n, const double *__restrict__ m,
                                                     const double *__restrict__ v, const double *__restrict__ e,
                                                     double *scratch) {
    __shared__ double sh[5][kBlock];
    double q[5] = {0, 0, 0, 0, 0};
    const int64_t base = (int64_t)blockIdx.x * kCellsPerBlock;
    for (int j = 0; j < kPerThread; ++j) {
        const int64_t c = base + (int64_t)j * kBlock + threadIdx.x;
        if (c < n) {
            const double mc = m[c];
            q[0] += mc;
            for (int a = 0; a < dim; ++a) q[1 + a] += mc * v[a * n + c];
            q[4] += mc * e[c];
        }
    }
    block_sum5(q, sh);
    if (threadIdx.x == 0)
        for (int i = 0; i < 5; ++i) scratch[blockIdx.x * kRow + i] = q[i];
}

__global__ void __launch_bounds__(kBlock) k_final(int nblocks, const double *scratch, double *out5) {
    __shared__ double sh[5][kBlock];
    double q[5] = {0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nblocks; b += kBlock)
        for (int i = 0; i < 5; ++i) q[i] += scratch[b * kRow + i];
    block_sum5(q, sh);
    if (threadIdx.x == 0)
        for (int i = 0; i < 5; ++i) out5[i] = q[i];
}

lmood_status scratch_for_current_device(double **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(LMOOD_ERR_CUDA, std::string("lmood_totals_noalloc: cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(LMOOD_ERR_ARG, "lmood_totals_noalloc: device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    // cudaGetSymbolAddress makes the device's primary context current if none is, so the
    // context id is read after the look-up on a first call and before it afterwards
    const unsigned long long ctx = g_scratch_ptr[dev] ? current_context_id() : 0;
    if (!g_scratch_ptr[dev] || ctx == 0 || ctx != g_scratch_ctx[dev]) {
        double *p = nullptr;
        e = cudaGetSymbolAddress((void **)&p, g_totals_scratch);
        if (e != cudaSuccess || !p)
            return fail(LMOOD_ERR_CUDA, std::string("lmood_totals_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_scratch_ptr[dev] = p;
        g_scratch_ctx[dev] = current_context_id();
    }
    *out = g_scratch_ptr[dev];
    return LMOOD_OK;
}

}  // namespace

extern "C" lmood_status lmood_totals_noalloc(int dim, int64_t n_cells, const double *m, const double *v,
                                             const double *e, double *out5, void *stream) {
    if (dim != 2 && dim != 3) return fail(LMOOD_ERR_ARG, "lmood_totals_noalloc: dim must be 2 or 3");
    if (!m || !v || !e || !out5) return fail(LMOOD_ERR_ARG, "lmood_totals_noalloc: NULL pointer");
    if (n_cells < 1) return fail(LMOOD_ERR_ARG, "lmood_totals_noalloc: n_cells must be positive");
    if (n_cells > kMaxCells)
        return fail(LMOOD_ERR_ARG, "lmood_totals_noalloc: n_cells " + std::to_string(n_cells) +
                                       " exceeds the no-allocation limit of " + std::to_string(kMaxCells) +
                                       " cells (use lmood_totals)");
    double *scratch = nullptr;
    lmood_status s = scratch_for_current_device(&scratch);
    if (s) return s;
    cudaStream_t st = (cudaStream_t)stream;
    const int nblocks = (int)((n_cells + kCellsPerBlock - 1) / kCellsPerBlock);
    k_partials<<<nblocks, kBlock, 0, st>>>(dim, n_cells, m, v, e, scratch);
    k_final<<<1, kBlock, 0, st>>>(nblocks, scratch, out5);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return fail(LMOOD_ERR_CUDA, std::string("lmood_totals_noalloc: launch: ") + cudaGetErrorString(err));
    return LMOOD_OK;
}
