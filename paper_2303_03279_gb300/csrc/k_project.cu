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
//
// Sessions whose metrics are all spectral project in the frequency domain instead: the taper
// and the band DFT act on the sample axis and M on the node axis, so the band spectra of the
// source trials are M times the band spectra of the sensor trials. The C sensor channels are
// transformed (k_spectrum, direct mode) and their spectra projected: 2 n C 2B flops per trial
// instead of 2 n C N (B band bins, N samples; 80 against 500 at 40 bins of 500-sample
// trials), the same GEMM tiling with the 2B real and imaginary parts as columns.
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

// Projected band spectra of trial blockIdx.z: columns 2 b + h of the product are the real
// (h = 0) and imaginary (h = 1) parts of bin b; written into the session's ring slot with its
// prescale.
__global__ void __launch_bounds__(256) k_project_spectra(const float* __restrict__ M, const float2* __restrict__ Xs,
                                                         float2* __restrict__ ring, int n, int C, int B,
                                                         int write_from, int slots, const FcCtrl* ctrl) {
    if (ctrl->bad) return;
    __shared__ float sm[TK][TM + 4];  // M tile, transposed: [k][row]
    __shared__ float sx[TK][TN + 4];  // spectra tile: [channel][2 bin + part]
    const int t = blockIdx.z;
    const float2* Xt = Xs + (size_t)t * B * C;
    const int r0 = blockIdx.y * TM, c0 = blockIdx.x * TN;  // c0: first column (even)
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int cols = 2 * B;
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    for (int k0 = 0; k0 < C; k0 += TK) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = tid + q * 256;
            const int mr = e / TK, mk = e % TK;
            const int gr = r0 + mr, gk = k0 + mk;
            sm[mk][mr] = (gr < n && gk < C) ? M[(size_t)gr * C + gk] : 0.f;
        }
#pragma unroll
        for (int q = 0; q < 2; ++q) {  // 16 channels x 32 bins of (re, im)
            const int e = tid + q * 256;
            const int xk = e / (TN / 2), xb = e % (TN / 2);
            const int hk = k0 + xk, b = c0 / 2 + xb;
            const float2 v = (hk < C && b < B) ? Xt[(size_t)b * C + hk] : make_float2(0.f, 0.f);
            sx[xk][2 * xb] = v.x;
            sx[xk][2 * xb + 1] = v.y;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < TK; ++k) {
            float a[4], bb[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = sm[k][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bb[j] = sx[k][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = __fmaf_rn(a[i], bb[j], acc[i][j]);
        }
        __syncthreads();
    }
    float scale = ctrl->scale;
    if (scale == 0.f) scale = 1.f;
    const int slot = (int)((ctrl->pushed + write_from + t) % slots);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int gr = r0 + ty * 4 + i;
        if (gr >= n) continue;
#pragma unroll
        for (int j = 0; j < 4; j += 2) {
            const int b = (c0 + tx * 4 + j) / 2;
            if (2 * b < cols)
                ring[((size_t)slot * B + b) * n + gr] = make_float2(__fmul_rn(acc[i][j], scale), __fmul_rn(acc[i][j + 1], scale));
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

cudaError_t launch_project_spectra(const float* M, const float2* Xs, float2* ring, int n, int C, int B, int count,
                                   int write_from, int slots, const FcCtrl* ctrl, cudaStream_t st) {
    if (n <= 0 || C <= 0 || B <= 0 || count <= 0 || count > 65535) return cudaErrorInvalidValue;
    dim3 grid((2 * B + TN - 1) / TN, (n + TM - 1) / TM, count);
    k_project_spectra<<<grid, 256, 0, st>>>(M, Xs, ring, n, C, B, write_from, slots, ctrl);
    return cudaGetLastError();
}
