// k_project.cu - source projection of sensor trials ahead of the spectrum.
//
// In the paper's source-level pipeline (Methods 2.5, Figure 1) every trial is mapped to
// the source space by the inverse operator (RTC-MNE) before the connectivity step:
// y_k = M x_k, M [n_sources][n_channels], x_k [n_channels][n_samples]. Here it is a
// batched FP32 GEMM on the CUDA cores: 2 n C N flops per trial, small beside the pair work
// (n^2 scaling) that follows, and in the time domain, so COR and XCOR see source signals.
//
// CTA: one 64 x 64 tile of Y (sources x samples) of one trial; 256 threads, 4 x 4 outputs
// each; the inner dimension in chunks of 16 staged in shared memory; FMA in a fixed order.
#include "fc_internal.h"

namespace {

constexpr int TM = 64, TN = 64, TK = 16;

__global__ void __launch_bounds__(256) k_project(const float* __restrict__ M, const float* __restrict__ X,
                                                 float* __restrict__ Y, int n, int C, int N) {
    __shared__ float sm[TK][TM + 4];  // M tile, transposed: [k][row]
    __shared__ float sx[TK][TN + 4];  // X tile: [k][col]
    const int trial = blockIdx.z;
    const float* Xk = X + (size_t)trial * C * N;
    float* Yk = Y + (size_t)trial * n * N;
    const int r0 = blockIdx.y * TM, c0 = blockIdx.x * TN;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    for (int k0 = 0; k0 < C; k0 += TK) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = tid + q * 256;  // 1024 elements per tile
            const int mr = e / TK, mk = e % TK;   // M: row, k
            const int xk = e / TN, xc = e % TN;   // X: k, col
            const int gr = r0 + mr, gk = k0 + mk;
            sm[mk][mr] = (gr < n && gk < C) ? M[(size_t)gr * C + gk] : 0.f;
            const int hk = k0 + xk, hc = c0 + xc;
            sx[xk][xc] = (hk < C && hc < N) ? Xk[(size_t)hk * N + hc] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < TK; ++k) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = sm[k][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = sx[k][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = __fmaf_rn(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int gr = r0 + ty * 4 + i;
        if (gr >= n) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gc = c0 + tx * 4 + j;
            if (gc < N) Yk[(size_t)gr * N + gc] = acc[i][j];
        }
    }
}

}  // namespace

cudaError_t launch_project(const float* M, const float* X, float* Y, int n, int C, int N, int count,
                           cudaStream_t st) {
    if (n <= 0 || C <= 0 || N <= 0 || count <= 0 || count > 65535) return cudaErrorInvalidValue;
    dim3 grid((N + TN - 1) / TN, (n + TM - 1) / TM, count);
    k_project<<<grid, 256, 0, st>>>(M, X, Y, n, C, N);
    return cudaGetLastError();
}
