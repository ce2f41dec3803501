// k_post.cu - network post-processing: normalization by the maximum edge weight, the
// strongest p % of the edges, node degree and node strength.
//
// Results 3.1.2 / 3.2.2: every network is normalized by its maximum edge weight; Results
// 3.2.2 / 3.2.3 and the figures show only the strongest 5 %, 10 % or 25 % of the edges;
// the Introduction names node degree and node strength as the graph measures drawn.
// Edges are ranked by magnitude (IMAGCOHY is signed); k = ceil(p P / 100) edges are kept,
// among equal magnitudes the lower packed index first; a NaN edge counts as 0; strength is
// the sum of a node's kept normalized magnitudes.
//
// Selection is a radix select on the magnitude's IEEE bits (monotone for non-negative
// floats): four passes of 8-bit histograms narrow the k-th largest key T; every key > T is
// kept, and of the keys equal to T the first (k - #greater) in index order, ranked by a
// scan over fixed contiguous chunks. Each pass reads the network once (4 B per edge).
// Degree and strength: one warp per node, its row of the packed triangle in a fixed order
// and a fixed reduction tree, so the floating-point sums are reproducible.
#include "fc_internal.h"

namespace {

constexpr int CHUNK = 4096;  // edges per block in the tie-rank passes (256 threads x 16)

__device__ __forceinline__ unsigned int mag_key(float w) {
    const unsigned int b = __float_as_uint(w) & 0x7fffffffu;
    return b > 0x7f800000u ? 0u : b;  // NaN counts as 0
}

__global__ void k_post_max(const float* __restrict__ w, long long P, PostState* st) {
    unsigned int m = 0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < P; e += (long long)gridDim.x * blockDim.x)
        m = max(m, mag_key(w[e]));
    for (int o = 16; o; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(&st->max_key, m);
}

__global__ void k_post_hist(const float* __restrict__ w, long long P, PostState* st, int shift) {
    __shared__ unsigned int h[256];
    for (int b = threadIdx.x; b < 256; b += blockDim.x) h[b] = 0;
    __syncthreads();
    const unsigned int prefix = st->prefix, mask = st->mask;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < P; e += (long long)gridDim.x * blockDim.x) {
        const unsigned int k = mag_key(w[e]);
        if ((k & mask) == prefix) atomicAdd(&h[(k >> shift) & 255u], 1u);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < 256; b += blockDim.x)
        if (h[b]) atomicAdd(&st->hist[b], (unsigned long long)h[b]);
}

// One block of 256 threads: the digit of the k_rem-th largest key among the candidates.
__global__ void k_post_pick(PostState* st, int shift) {
    __shared__ unsigned long long above[256];  // candidates in digits > b
    __shared__ unsigned long long kr_s;
    const int b = threadIdx.x;
    unsigned long long s = 0;
    for (int c = b + 1; c < 256; ++c) s += st->hist[c];
    above[b] = s;
    if (b == 0) kr_s = (unsigned long long)st->k_rem;  // read before the one writer below
    __syncthreads();
    const unsigned long long kr = kr_s;
    if (above[b] < kr && above[b] + st->hist[b] >= kr) {
        st->k_rem = (long long)(kr - above[b]);
        st->prefix |= (unsigned int)b << shift;
        st->mask |= 255u << shift;
    }
    __syncthreads();
    st->hist[b] = 0;
}

__global__ void k_post_tiecount(const float* __restrict__ w, long long P, const PostState* st,
                                unsigned long long* __restrict__ ties) {
    __shared__ unsigned int cnt;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    const unsigned int T = st->prefix;
    const long long e0 = (long long)blockIdx.x * CHUNK + threadIdx.x * 16;
    unsigned int c = 0;
    for (int q = 0; q < 16; ++q) {
        const long long e = e0 + q;
        if (e < P && mag_key(w[e]) == T) ++c;
    }
    atomicAdd(&cnt, c);
    __syncthreads();
    if (threadIdx.x == 0) ties[blockIdx.x] = cnt;
}

// Exclusive scan of the per-chunk tie counts (one block of 1024 threads, serial carry).
__global__ void k_post_tiescan(unsigned long long* ties, long long nchunks) {
    __shared__ unsigned long long s[1024];
    __shared__ unsigned long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (long long base = 0; base < nchunks; base += 1024) {
        const long long i = base + threadIdx.x;
        const unsigned long long v = i < nchunks ? ties[i] : 0ull;
        s[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {  // inclusive Hillis-Steele scan
            const unsigned long long add = threadIdx.x >= o ? s[threadIdx.x - o] : 0ull;
            __syncthreads();
            s[threadIdx.x] += add;
            __syncthreads();
        }
        if (i < nchunks) ties[i] = carry + s[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry += s[1023];
        __syncthreads();
    }
}

__global__ void k_post_mark(const float* __restrict__ w, long long P, const PostState* st,
                            const unsigned long long* __restrict__ tieoff, float* __restrict__ out,
                            unsigned char* __restrict__ keep) {
    __shared__ unsigned int ts[256];
    const unsigned int T = st->prefix;
    const unsigned long long need = (unsigned long long)st->k_rem;
    const bool none = st->k_total == 0;
    const float mx = __uint_as_float(st->max_key);
    const long long e0 = (long long)blockIdx.x * CHUNK + threadIdx.x * 16;
    unsigned int keys[16];
    unsigned int c = 0;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        const long long e = e0 + q;
        keys[q] = e < P ? mag_key(w[e]) : 0u;
        c += (e < P && keys[q] == T) ? 1u : 0u;
    }
    ts[threadIdx.x] = c;
    __syncthreads();
    for (int o = 1; o < 256; o <<= 1) {
        const unsigned int add = threadIdx.x >= o ? ts[threadIdx.x - o] : 0u;
        __syncthreads();
        ts[threadIdx.x] += add;
        __syncthreads();
    }
    unsigned long long rank = tieoff[blockIdx.x] + ts[threadIdx.x] - c;  // ties before this thread's first
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        const long long e = e0 + q;
        if (e >= P) break;
        bool k = false;
        if (!none) {
            if (keys[q] > T) {
                k = true;
            } else if (keys[q] == T) {
                k = rank < need;
                ++rank;
            }
        }
        keep[e] = k ? 1 : 0;
        const float v = w[e];
        out[e] = (k && mx > 0.f && keys[q] != 0u) ? __fdiv_rn(v, mx) : 0.f;
    }
}

__device__ __forceinline__ long long tri_index(int i, int j, int n) {  // i < j
    return (long long)i * n - (long long)i * (i + 1) / 2 + (j - i - 1);
}

__global__ void k_post_nodes(const float* __restrict__ out, const unsigned char* __restrict__ keep, int n,
                             int* __restrict__ degree, float* __restrict__ strength) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= n) return;
    const int i = warp;
    int d = 0;
    double s = 0.0;  // FP64 partial sums: their rounding stays far below the FP32 result's
    for (int j = lane; j < n; j += 32) {
        if (j == i) continue;
        const long long e = i < j ? tri_index(i, j, n) : tri_index(j, i, n);
        if (keep[e]) {
            ++d;
            s += (double)fabsf(out[e]);
        }
    }
    for (int o = 16; o; o >>= 1) {
        d += __shfl_xor_sync(0xffffffffu, d, o);
        s += __shfl_xor_sync(0xffffffffu, s, o);
    }
    if (lane == 0) {
        degree[i] = d;
        strength[i] = (float)s;
    }
}

}  // namespace

size_t post_scratch_bytes(long long P) {
    const long long nchunks = (P + CHUNK - 1) / CHUNK;
    return sizeof(PostState) + (size_t)nchunks * 8 + (size_t)P + 256;
}

cudaError_t launch_network_top(const float* w, long long P, int n, long long k, void* scratch, float* out,
                               int* degree, float* strength, int num_sms, cudaStream_t stream) {
    if (P <= 0) return cudaSuccess;
    PostState* st = static_cast<PostState*>(scratch);
    const long long nchunks = (P + CHUNK - 1) / CHUNK;
    unsigned long long* ties = reinterpret_cast<unsigned long long*>(static_cast<char*>(scratch) + sizeof(PostState));
    unsigned char* keep = reinterpret_cast<unsigned char*>(ties + nchunks);
    PostState init{};
    init.k_rem = k;
    init.k_total = k;
    cudaError_t e = cudaMemcpyAsync(st, &init, sizeof(PostState), cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess) return e;
    const int grid = 4 * num_sms;
    k_post_max<<<grid, 256, 0, stream>>>(w, P, st);
    for (int pass = 0; pass < 4 && k > 0; ++pass) {
        const int shift = 24 - 8 * pass;
        k_post_hist<<<grid, 256, 0, stream>>>(w, P, st, shift);
        k_post_pick<<<1, 256, 0, stream>>>(st, shift);
    }
    k_post_tiecount<<<(unsigned)nchunks, 256, 0, stream>>>(w, P, st, ties);
    k_post_tiescan<<<1, 1024, 0, stream>>>(ties, nchunks);
    k_post_mark<<<(unsigned)nchunks, 256, 0, stream>>>(w, P, st, ties, out, keep);
    if (degree && strength) k_post_nodes<<<(n * 32 + 255) / 256, 256, 0, stream>>>(out, keep, n, degree, strength);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(stream);
}
