/*
 * Plain-C use of libnf's C ABI (include/nf.h): no Python, no torch.
 * Allocates device memory with the CUDA runtime, bins a small uniform box,
 * computes near-field accelerations, the adjoint and the far field, and
 * prints a summary line that the test compares with its own expectations.
 *
 * Build (see tests/test_gpu_c_abi.py):
 *   gcc -O2 -I include tests/c_abi/nf_c_example.c -o nf_c_example \
 *       -L paper_2110_11392_gb300 -lnf -L /usr/local/cuda/lib64 -lcudart -Wl,-rpath,...
 */
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include "nf.h"

static unsigned long long lcg = 88172645463325252ULL;
static float uniform01(void)
{
    lcg = lcg * 6364136223846793005ULL + 1442695040888963407ULL;
    return (float)((lcg >> 40) * (1.0 / 16777216.0));
}

#define CHECK_CUDA(x)                                                               \
    do {                                                                            \
        cudaError_t e_ = (x);                                                       \
        if (e_ != cudaSuccess) {                                                    \
            fprintf(stderr, "%s: %s\n", #x, cudaGetErrorString(e_));                \
            return 2;                                                               \
        }                                                                           \
    } while (0)

#define CHECK_NF(x)                                                                 \
    do {                                                                            \
        int r_ = (x);                                                               \
        if (r_ != NF_OK) {                                                          \
            fprintf(stderr, "%s: status %d: %s\n", #x, r_, nf_last_error());         \
            return 3;                                                               \
        }                                                                           \
    } while (0)

int main(void)
{
    const int64_t N = 20000;
    const int K = 7, R = 2;
    const double box = 1.0, eps = 1.0 / (40.0 * cbrt((double)N));
    float *h_pos = (float *)malloc(sizeof(float) * 3 * N);
    float *h_acc = (float *)malloc(sizeof(float) * 3 * N);
    for (int64_t i = 0; i < 3 * N; ++i) {
        float u = uniform01();
        h_pos[i] = u < 1.0f ? u : 0.0f;
    }
    float *pos, *acc, *g, *grad;
    double *net;
    void *ws;
    size_t ws_bytes = nf_workspace_bytes(N, K, R);
    if (ws_bytes == 0) {
        fprintf(stderr, "nf_workspace_bytes: %s\n", nf_last_error());
        return 1;
    }
    CHECK_CUDA(cudaMalloc((void **)&pos, sizeof(float) * 3 * N));
    CHECK_CUDA(cudaMalloc((void **)&acc, sizeof(float) * 3 * N));
    CHECK_CUDA(cudaMalloc((void **)&g, sizeof(float) * 3 * N));
    CHECK_CUDA(cudaMalloc((void **)&grad, sizeof(float) * 3 * N));
    CHECK_CUDA(cudaMalloc((void **)&net, sizeof(double) * 3));
    CHECK_CUDA(cudaMalloc(&ws, ws_bytes));
    cudaStream_t s;
    CHECK_CUDA(cudaStreamCreate(&s));
    CHECK_CUDA(cudaMemcpyAsync(pos, h_pos, sizeof(float) * 3 * N, cudaMemcpyHostToDevice, s));

    /* a rejected call launches nothing and says why */
    int bad = nf_forces(pos, N, box, 4, R, eps, acc, NULL, ws, ws_bytes, s);
    if (bad != NF_ERR_ARG) return 4;

    CHECK_NF(nf_forces(pos, N, box, K, R, eps, acc, net, ws, ws_bytes, s));
    CHECK_NF(nf_status_read(ws, s));
    int64_t stats[4];
    CHECK_NF(nf_stats_read(ws, stats, s));
    double h_net[3];
    CHECK_CUDA(cudaMemcpy(h_acc, acc, sizeof(float) * 3 * N, cudaMemcpyDeviceToHost));
    CHECK_CUDA(cudaMemcpy(h_net, net, sizeof(double) * 3, cudaMemcpyDeviceToHost));
    double sum_abs = 0.0;
    for (int64_t i = 0; i < 3 * N; ++i) sum_abs += fabs((double)h_acc[i]);

    /* adjoint with g = acc: grad = dL/dx for L = sum |a|^2 / 2 */
    CHECK_CUDA(cudaMemcpyAsync(g, acc, sizeof(float) * 3 * N, cudaMemcpyDeviceToDevice, s));
    CHECK_NF(nf_forces_adjoint(pos, g, N, box, K, R, eps, grad, ws, ws_bytes, s));
    CHECK_NF(nf_status_read(ws, s));

    /* far field at order 4: derivatives once, then the far accelerations in FP64 */
    const int p = 4;
    void *derivs, *wsf;
    double *far;
    const size_t d_bytes = nf_derivatives_bytes(K, p), f_bytes = nf_far_workspace_bytes(N, K, p);
    if (d_bytes == 0 || f_bytes == 0) return 5;
    CHECK_CUDA(cudaMalloc(&derivs, d_bytes));
    CHECK_CUDA(cudaMalloc(&wsf, f_bytes));
    CHECK_CUDA(cudaMalloc((void **)&far, sizeof(double) * 3 * N));
    CHECK_NF(nf_derivatives(K, R, p, box, derivs, d_bytes, wsf, f_bytes, s));
    CHECK_NF(nf_far_forces(pos, N, box, K, R, p, derivs, d_bytes, far, NULL, NULL, wsf, f_bytes, s));
    CHECK_NF(nf_status_read(wsf, s));
    double h_far[3];
    CHECK_CUDA(cudaMemcpy(h_far, far, sizeof(double) * 3, cudaMemcpyDeviceToHost));
    CHECK_NF(nf_far_release());

    printf("ok N=%lld pairs=%lld items=%lld maxocc=%lld net=%.3e mean_abs_acc=%.6e acc0=%.9e %.9e %.9e "
           "far0=%.15e %.15e %.15e\n",
           (long long)N, (long long)stats[0], (long long)stats[1], (long long)stats[2],
           fmax(fabs(h_net[0]), fmax(fabs(h_net[1]), fabs(h_net[2]))), sum_abs / (3.0 * N),
           h_acc[0], h_acc[1], h_acc[2], h_far[0], h_far[1], h_far[2]);
    cudaFree(derivs);
    cudaFree(wsf);
    cudaFree(far);
    cudaFree(pos);
    cudaFree(acc);
    cudaFree(g);
    cudaFree(grad);
    cudaFree(net);
    cudaFree(ws);
    cudaStreamDestroy(s);
    free(h_pos);
    free(h_acc);
    return 0;
}
