// k_cor.cu - correlation (COR), Supplementary Information 1 (Time Domain), and Methods
// 2.4 ("a simple dot product and division by the number of samples"): the per-trial
// normalization and the combination of trial-group partial sums. The products themselves
// run on the tensor cores (k_cor_tc.cu).
//
// Per trial k and node i: z_i = (x_i - mean x_i) / ||x_i - mean x_i|| (0 for a constant
// node), so COR_k(i, j) = z_i . z_j; the network is the mean over the window's trials.
#include "df32.cuh"
#include "fc_internal.h"
#include "row_stats.cuh"

namespace {

// One warp per (trial, node): mean and norm as double words on the FP32 pipes (row_stats.cuh),
// z = deviation / norm in FP32 (0 for a constant node).
__global__ void k_cor_normalize(CorArgs a) {
    const FcCtrl* c = a.ctrl;
    if (c->bad) return;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int ntr = a.count - a.write_from;
    if (warp >= ntr * a.n) return;
    const int tr = a.write_from + warp / a.n, node = warp % a.n;
    const float* x = a.x + ((size_t)tr * a.n + node) * a.N;
    const RowStats st = warp_row_stats(x, a.N, lane);
    const float inv = st.ss > 0.f ? __fdiv_rn(1.0f, __fsqrt_rn(st.ss)) : 0.f;
    const long long g = c->pushed + tr;
    float* z = a.zring + ((size_t)(g % a.slots) * a.n + node) * a.N;
    for (int t = lane; t < a.N; t += 32) z[t] = __fmul_rn(st.dev(x[t]), inv);
}

// Sum of the trial groups' double-float partial sums, in group order.
__global__ void k_cor_combine(CorArgs a) {
    const FcCtrl* c = a.ctrl;
    if (c->bad) return;
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.P) return;
    const long long end = c->pushed + a.count;
    const long long start = (a.W > 0 && end > a.W) ? end - a.W : 0;
    const int K = (int)(end - start);
    df32 acc = df_make(0.f, 0.f);
    for (int g = 0; g < a.groups; ++g)
        acc = df_add_df(acc, df_make(a.part[(2 * (size_t)g) * a.P + p], a.part[(2 * (size_t)g + 1) * a.P + p]));
    a.cor_acc[p] = acc.hi;
    a.cor_acc[a.P + p] = acc.lo;
    if (a.finalize) a.net[p] = __fmul_rn(df_to_f(acc), 1.0f / (float)K);
}

}  // namespace

cudaError_t launch_cor_combine(const CorArgs& a, cudaStream_t st) {
    k_cor_combine<<<(unsigned)((a.P + 255) / 256), 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_cor_normalize(const CorArgs& a, cudaStream_t st) {
    const long long warps = (long long)(a.count - a.write_from) * a.n;
    if (warps <= 0) return cudaSuccess;
    k_cor_normalize<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, st>>>(a);
    return cudaGetLastError();
}
