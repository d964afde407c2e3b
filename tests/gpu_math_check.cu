// Test helper: evaluates the step's FP64 scalar functions of J next to CUDA's own log / rcbrt
// on the device, so that the tests can bound their difference. Compiled by the test.
#include "lmood_dev.cuh"

__global__ void k_eval(const double *J, int n, double *lg, double *lg_ref, double *rc, double *rc_ref) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    lg[i] = lmood::log_j(J[i]);
    lg_ref[i] = log(J[i]);
    rc[i] = lmood::rcbrt_j(J[i]);
    rc_ref[i] = rcbrt(J[i]);
}

extern "C" int eval_math(const double *J_host, int n, double *out_host /* [4][n] */) {
    double *d;
    if (cudaMalloc(&d, sizeof(double) * 5 * n) != cudaSuccess) return 1;
    cudaMemcpy(d, J_host, sizeof(double) * n, cudaMemcpyHostToDevice);
    k_eval<<<(n + 255) / 256, 256>>>(d, n, d + n, d + 2 * n, d + 3 * n, d + 4 * n);
    cudaError_t e = cudaMemcpy(out_host, d + n, sizeof(double) * 4 * n, cudaMemcpyDeviceToHost);
    cudaFree(d);
    return e == cudaSuccess ? 0 : 2;
}

// order keys: for pairs (a[i], b[i]) the key comparisons and the min / max through the keys,
// next to the FP64 ones
__global__ void k_keys(const double *a, const double *b, int n, int *ge, int *ge_ref, double *mn, double *mx) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const long long ka = lmood::order_key(a[i]), kb = lmood::order_key(b[i]);
    ge[i] = ka >= kb;
    ge_ref[i] = a[i] >= b[i];
    mn[i] = lmood::key_value(min(ka, kb));
    mx[i] = lmood::key_value(max(ka, kb));
}

extern "C" int eval_keys(const double *a_host, const double *b_host, int n, int *ge_host /* [2][n] */,
                         double *mm_host /* [2][n] */) {
    double *d;
    int *di;
    if (cudaMalloc(&d, sizeof(double) * 4 * n) != cudaSuccess) return 1;
    if (cudaMalloc(&di, sizeof(int) * 2 * n) != cudaSuccess) {
        cudaFree(d);
        return 1;
    }
    cudaMemcpy(d, a_host, sizeof(double) * n, cudaMemcpyHostToDevice);
    cudaMemcpy(d + n, b_host, sizeof(double) * n, cudaMemcpyHostToDevice);
    k_keys<<<(n + 255) / 256, 256>>>(d, d + n, n, di, di + n, d + 2 * n, d + 3 * n);
    cudaError_t e = cudaMemcpy(mm_host, d + 2 * n, sizeof(double) * 2 * n, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(ge_host, di, sizeof(int) * 2 * n, cudaMemcpyDeviceToHost);
    cudaFree(d);
    cudaFree(di);
    return e == cudaSuccess ? 0 : 2;
}
