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
