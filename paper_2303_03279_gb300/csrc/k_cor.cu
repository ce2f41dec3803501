// k_cor.cu - correlation (COR), Supplementary Information 1 (Time Domain), and Methods
// 2.4 ("a simple dot product and division by the number of samples").
//
// Per trial k and node i: z_i = (x_i - mean x_i) / ||x_i - mean x_i|| (0 for a constant
// node), so COR_k(i, j) = z_i . z_j. The network is the mean over the window's trials.
// The products form a symmetric rank-N update (SYRK) over the upper triangle: 64 x 64
// node tiles, 4 x 4 register micro-tiles, samples staged through shared memory. Each
// trial's dot product is summed in FP32 in a fixed order (per 32-sample chunk, then
// across chunks) and the per-trial values enter a double-float running sum, so the
// value subtracted when a trial leaves the window has exactly the bits that were added.
#include "df32.cuh"
#include "fc_internal.h"

namespace {

constexpr int CT = 64;  // nodes per tile
constexpr int CK = 32;  // samples per chunk

__device__ __forceinline__ long long packed_index(int i, int j, int n) {
    return (long long)i * n - (long long)i * (i + 1) / 2 + (j - i - 1);
}

// One warp per (trial, node): mean and norm in FP64, z in FP32.
__global__ void k_cor_normalize(CorArgs a) {
    const FcCtrl* c = a.ctrl;
    if (c->bad) return;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int ntr = a.count - a.write_from;
    if (warp >= ntr * a.n) return;
    const int tr = a.write_from + warp / a.n, node = warp % a.n;
    const float* x = a.x + ((size_t)tr * a.n + node) * a.N;
    double s = 0.0;
    for (int t = lane; t < a.N; t += 32) s += (double)x[t];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    const double mean = s / a.N;
    double q = 0.0;
    for (int t = lane; t < a.N; t += 32) {
        const double d = (double)x[t] - mean;
        q += d * d;
    }
    for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
    const double inv = q > 0.0 ? 1.0 / sqrt(q) : 0.0;
    const long long g = c->pushed + tr;
    float* z = a.zring + ((size_t)(g % a.slots) * a.n + node) * a.N;
    for (int t = lane; t < a.N; t += 32) z[t] = (float)(((double)x[t] - mean) * inv);
}

__device__ __forceinline__ void tile_of(int tp, int nt, int& ta, int& tb) {
    int r = tp, a = 0;
    while (r >= nt - a) {
        r -= nt - a;
        ++a;
    }
    ta = a;
    tb = a + r;
}

// Dot products z_i^k . z_j^k of one trial for this thread's 4 x 4 pairs.
__device__ __forceinline__ void trial_dots(const float* __restrict__ z, int n, int N, int ta, int tb,
                                           float (*As)[CT + 4], float (*Bs)[CT + 4], float d[4][4]) {
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int q = 0; q < 4; ++q) d[r][q] = 0.f;
    for (int t0 = 0; t0 < N; t0 += CK) {
        __syncthreads();
        for (int e = tid; e < CT * CK; e += 256) {
            const int r = e / CK, t = e % CK;
            const int ni = ta * CT + r, nj = tb * CT + r;
            const bool tv = t0 + t < N;
            As[t][r] = (ni < n && tv) ? z[(size_t)ni * N + t0 + t] : 0.f;
            Bs[t][r] = (nj < n && tv) ? z[(size_t)nj * N + t0 + t] : 0.f;
        }
        __syncthreads();
        float p[4][4];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int q = 0; q < 4; ++q) p[r][q] = 0.f;
#pragma unroll 8
        for (int t = 0; t < CK; ++t) {
            const float4 ra = *reinterpret_cast<const float4*>(&As[t][ty * 4]);
            const float4 rb = *reinterpret_cast<const float4*>(&Bs[t][tx * 4]);
            const float av[4] = {ra.x, ra.y, ra.z, ra.w};
            const float bv[4] = {rb.x, rb.y, rb.z, rb.w};
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int q = 0; q < 4; ++q) p[r][q] = __fmaf_rn(av[r], bv[q], p[r][q]);
        }
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int q = 0; q < 4; ++q) d[r][q] = __fadd_rn(d[r][q], p[r][q]);
    }
}

__global__ void __launch_bounds__(256) k_cor_update(CorArgs a) {
    const FcCtrl* c = a.ctrl;
    if (c->bad) return;
    const long long end = c->pushed + a.count;
    const long long start = (a.W > 0 && end > a.W) ? end - a.W : 0;
    const int K = (int)(end - start);
    const int nt = (a.n + CT - 1) / CT;
    int ta, tb;
    tile_of(blockIdx.x, nt, ta, tb);
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    __shared__ __align__(16) float As[CK][CT + 4];
    __shared__ __align__(16) float Bs[CK][CT + 4];

    long long idx[4][4];
    bool ok[4][4];
    df32 acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int i = ta * CT + ty * 4 + r, j = tb * CT + tx * 4 + q;
            ok[r][q] = i < j && j < a.n;
            idx[r][q] = ok[r][q] ? packed_index(i, j, a.n) : 0;
            acc[r][q] = df_make(0.f, 0.f);
            if (a.mode == 0 && ok[r][q]) acc[r][q] = df_make(a.cor_acc[idx[r][q]], a.cor_acc[a.P + idx[r][q]]);
        }
    float d[4][4];
    if (a.mode == 0) {
        // stream: add the newest trial, subtract the one leaving the window
        const long long tn = end - 1;
        trial_dots(a.zring + (size_t)(tn % a.slots) * a.n * a.N, a.n, a.N, ta, tb, As, Bs, d);
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[r][q] = df_add_f(acc[r][q], d[r][q]);
        if (a.W > 0 && tn >= a.W) {
            const long long to = tn - a.W;
            trial_dots(a.zring + (size_t)(to % a.slots) * a.n * a.N, a.n, a.N, ta, tb, As, Bs, d);
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[r][q] = df_add_f(acc[r][q], -d[r][q]);
        }
    } else {
        for (long long k = start; k < end; ++k) {
            trial_dots(a.zring + (size_t)(k % a.slots) * a.n * a.N, a.n, a.N, ta, tb, As, Bs, d);
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[r][q] = df_add_f(acc[r][q], d[r][q]);
        }
    }
    const float invK = 1.0f / (float)K;
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (!ok[r][q]) continue;
            a.cor_acc[idx[r][q]] = acc[r][q].hi;
            a.cor_acc[a.P + idx[r][q]] = acc[r][q].lo;
            if (a.finalize) a.net[idx[r][q]] = __fmul_rn(df_to_f(acc[r][q]), invK);
        }
}

}  // namespace

cudaError_t launch_cor_normalize(const CorArgs& a, cudaStream_t st) {
    const long long warps = (long long)(a.count - a.write_from) * a.n;
    if (warps <= 0) return cudaSuccess;
    k_cor_normalize<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_cor_update(const CorArgs& a, cudaStream_t st) {
    const int nt = (a.n + CT - 1) / CT;
    k_cor_update<<<nt * (nt + 1) / 2, 256, 0, st>>>(a);
    return cudaGetLastError();
}
