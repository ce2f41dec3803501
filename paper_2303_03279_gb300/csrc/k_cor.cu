// k_cor.cu - correlation (COR), Supplementary Information 1 (Time Domain), and Methods
// 2.4 ("a simple dot product and division by the number of samples").
//
// Per trial k and node i: z_i = (x_i - mean x_i) / ||x_i - mean x_i|| (0 for a constant
// node), so COR_k(i, j) = z_i . z_j. The network is the mean over the window's trials.
// The products form a symmetric rank-N update (SYRK) over the upper triangle: 64 x 64
// node tiles, 4 x 4 register micro-tiles, samples staged through swizzled, double-buffered
// shared memory. Each
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

// Shared tiles [t][row], unpadded, rows XOR-swizzled by the sample's 4-group: the staging
// stores (4 rows x 8 float4 per warp) hit 32 distinct banks and the compute's float4 reads
// of 4 consecutive rows stay aligned and in order.
__device__ __forceinline__ int swz(int t, int r) { return r ^ (((t >> 2) & 7) << 2); }

// This thread's share of one chunk of one tile: rows (tid >> 3) and (tid >> 3) + 32, samples
// t0 + 4 (tid & 7) .. + 3 (float4 along the row when N % 4 == 0).
__device__ __forceinline__ void load_chunk(const float* __restrict__ z, int n, int N, int tile, int t0, float4 v[2]) {
    const int tid = threadIdx.x, t = t0 + 4 * (tid & 7);
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int row = tile * CT + (tid >> 3) + 32 * q;
        float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
        if (row < n) {
            const float* zr = z + (size_t)row * N;
            if ((N & 3) == 0 && t + 3 < N) {
                x = *reinterpret_cast<const float4*>(zr + t);
            } else {
                if (t < N) x.x = zr[t];
                if (t + 1 < N) x.y = zr[t + 1];
                if (t + 2 < N) x.z = zr[t + 2];
                if (t + 3 < N) x.w = zr[t + 3];
            }
        }
        v[q] = x;
    }
}
__device__ __forceinline__ void store_chunk(float (*S)[CT], const float4 v[2]) {
    const int tid = threadIdx.x, t = 4 * (tid & 7);
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int r = (tid >> 3) + 32 * q;
        S[t + 0][swz(t + 0, r)] = v[q].x;
        S[t + 1][swz(t + 1, r)] = v[q].y;
        S[t + 2][swz(t + 2, r)] = v[q].z;
        S[t + 3][swz(t + 3, r)] = v[q].w;
    }
}

// Dot products z_i^k . z_j^k of one trial for this thread's 4 x 4 pairs: FP32 per 32-sample
// chunk, the chunks added in order. Chunks are double-buffered: the next chunk is read into
// registers while this one is multiplied.
__device__ __forceinline__ void trial_dots(const float* __restrict__ z, int n, int N, int ta, int tb,
                                           float (*As)[CK][CT], float (*Bs)[CK][CT], float d[4][4]) {
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int q = 0; q < 4; ++q) d[r][q] = 0.f;
    const int nchunk = (N + CK - 1) / CK;
    float4 va[2], vb[2];
    load_chunk(z, n, N, ta, 0, va);
    load_chunk(z, n, N, tb, 0, vb);
    __syncthreads();  // the previous user of the buffers is done
    store_chunk(As[0], va);
    store_chunk(Bs[0], vb);
    __syncthreads();
    for (int ch = 0; ch < nchunk; ++ch) {
        const int cb = ch & 1;
        if (ch + 1 < nchunk) {
            load_chunk(z, n, N, ta, (ch + 1) * CK, va);
            load_chunk(z, n, N, tb, (ch + 1) * CK, vb);
        }
        float p[4][4];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int q = 0; q < 4; ++q) p[r][q] = 0.f;
#pragma unroll 8
        for (int t = 0; t < CK; ++t) {
            const float4 ra = *reinterpret_cast<const float4*>(&As[cb][t][swz(t, ty * 4)]);
            const float4 rb = *reinterpret_cast<const float4*>(&Bs[cb][t][swz(t, tx * 4)]);
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
        if (ch + 1 < nchunk) {  // the other buffer was last read before the previous barrier
            store_chunk(As[cb ^ 1], va);
            store_chunk(Bs[cb ^ 1], vb);
        }
        __syncthreads();
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
    __shared__ __align__(16) float As[2][CK][CT];
    __shared__ __align__(16) float Bs[2][CK][CT];

    // pair (i, j) of micro-tile entry (r, q); recomputed where needed to spare registers
    const int i0 = ta * CT + ty * 4, j0 = tb * CT + tx * 4;
    df32 acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int i = i0 + r, j = j0 + q;
            acc[r][q] = df_make(0.f, 0.f);
            if (a.mode == 0 && i < j && j < a.n) {
                const long long id = packed_index(i, j, a.n);
                acc[r][q] = df_make(a.cor_acc[id], a.cor_acc[a.P + id]);
            }
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
        // this CTA's share of the window's trials (several groups when tile pairs are few)
        const int tg = (K + a.groups - 1) / a.groups;
        const long long k0 = start + (long long)blockIdx.y * tg;
        const long long k1 = k0 + tg < end ? k0 + tg : end;
        for (long long k = k0; k < k1; ++k) {
            trial_dots(a.zring + (size_t)(k % a.slots) * a.n * a.N, a.n, a.N, ta, tb, As, Bs, d);
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[r][q] = df_add_f(acc[r][q], d[r][q]);
        }
    }
    const float invK = 1.0f / (float)K;
    const bool partial = a.mode == 1 && a.groups > 1;
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int i = i0 + r, j = j0 + q;
            if (!(i < j && j < a.n)) continue;
            const long long id = packed_index(i, j, a.n);
            if (partial) {
                a.part[(2 * (size_t)blockIdx.y) * a.P + id] = acc[r][q].hi;
                a.part[(2 * (size_t)blockIdx.y + 1) * a.P + id] = acc[r][q].lo;
                continue;
            }
            a.cor_acc[id] = acc[r][q].hi;
            a.cor_acc[a.P + id] = acc[r][q].lo;
            if (a.finalize) a.net[id] = __fmul_rn(df_to_f(acc[r][q]), invK);
        }
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

cudaError_t launch_cor_update(const CorArgs& a, cudaStream_t st) {
    const int nt = (a.n + CT - 1) / CT;
    if (a.groups < 1 || (a.groups > 1 && (a.mode != 1 || !a.part))) return cudaErrorInvalidValue;
    k_cor_update<<<dim3(nt * (nt + 1) / 2, a.mode == 1 ? a.groups : 1), 256, 0, st>>>(a);
    return cudaGetLastError();
}
