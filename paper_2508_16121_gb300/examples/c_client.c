/* A plain C client of libsvdlut: no PyTorch, only the CUDA runtime for
 * device memory.  It runs svdlut_apply on a 48 x 64 float image with all LUT
 * factors and weights zero, no grids and per-channel biases (0.25, 0.5, 0.75),
 * so every output pixel of channel c must equal that bias (Eq. 5 with
 * w = 0), and prints "c_client: ok" on success.  Exit status: 0 on success, 1
 * on a wrong value, 2 on an API or CUDA error. */
#include <cuda_runtime_api.h>
#include <stdio.h>
#include <stdlib.h>

#include "svdlut.h"

#define CHECK_CUDA(e)                                                           \
    do {                                                                        \
        cudaError_t err_ = (e);                                                 \
        if (err_ != cudaSuccess) {                                              \
            fprintf(stderr, "c_client: %s\n", cudaGetErrorString(err_));        \
            return 2;                                                           \
        }                                                                       \
    } while (0)

int main(void)
{
    const int H = 48, W = 64, D = 33, R = 8;
    const size_t npx = (size_t)3 * H * W;
    const float bias[3] = {0.25f, 0.5f, 0.75f};
    svdlut_dims dims = {D, R, 0, 2, 2, 2};
    float *x = NULL, *y = NULL, *U = NULL, *S = NULL, *V = NULL, *lw = NULL;
    float *hx = (float *)malloc(npx * sizeof(float)), *hy = (float *)malloc(npx * sizeof(float));
    float hlw[12] = {0};
    if (!hx || !hy) return 2;
    for (size_t i = 0; i < npx; ++i) hx[i] = (float)(i % 97) / 96.0f;
    for (int c = 0; c < 3; ++c) hlw[4 * c + 3] = bias[c];
    CHECK_CUDA(cudaMalloc((void **)&x, npx * sizeof(float)));
    CHECK_CUDA(cudaMalloc((void **)&y, npx * sizeof(float)));
    CHECK_CUDA(cudaMalloc((void **)&U, 9 * D * R * sizeof(float)));
    CHECK_CUDA(cudaMalloc((void **)&S, 9 * R * sizeof(float)));
    CHECK_CUDA(cudaMalloc((void **)&V, 9 * D * R * sizeof(float)));
    CHECK_CUDA(cudaMalloc((void **)&lw, 12 * sizeof(float)));
    CHECK_CUDA(cudaMemset(U, 0, 9 * D * R * sizeof(float)));
    CHECK_CUDA(cudaMemset(S, 0, 9 * R * sizeof(float)));
    CHECK_CUDA(cudaMemset(V, 0, 9 * D * R * sizeof(float)));
    CHECK_CUDA(cudaMemcpy(lw, hlw, sizeof hlw, cudaMemcpyHostToDevice));
    CHECK_CUDA(cudaMemcpy(x, hx, npx * sizeof(float), cudaMemcpyHostToDevice));
    svdlut_params p = {U, S, V, lw, NULL, NULL, NULL, NULL};
    svdlut_status st = svdlut_apply(&dims, &p, 1, H, W, SVDLUT_F32, x, y, NULL);
    if (st != SVDLUT_OK) {
        fprintf(stderr, "c_client: svdlut_apply: %s\n", svdlut_last_error());
        return 2;
    }
    CHECK_CUDA(cudaMemcpy(hy, y, npx * sizeof(float), cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < npx; ++i) {
        const float want = bias[i / ((size_t)H * W)];
        if (hy[i] != want) {
            fprintf(stderr, "c_client: y[%zu] = %g, want %g\n", i, hy[i], want);
            return 1;
        }
    }
    cudaFree(x);
    cudaFree(y);
    cudaFree(U);
    cudaFree(S);
    cudaFree(V);
    cudaFree(lw);
    free(hx);
    free(hy);
    printf("c_client: ok (%s)\n", svdlut_version());
    return 0;
}
