// k_spectrum.cu - per-trial taper + band spectrum (Methods 2.4: "for each trial, the
// frequency spectrum ... is calculated"), plus push validation and commit.
//
// X_i(f) = sum_{t < N} x_i(t) w(t) exp(-2 pi i f t / nfft) for the band bins f only: a
// real [n x N] by complex [N x B] product against a taper-folded factor table built on
// the host in FP64 (angle reduced exactly as (f t) mod nfft, then rounded to FP32).
// A band of B bins needs N*B complex factors per node: cheaper than a full real FFT for
// the narrow bands of the paper (4 to 101 bins) and a plain dense contraction. The
// contraction runs in FP32 on the CUDA cores: the tensor-core formats (TF32/BF16) would
// put a 1e-3 relative error into every spectrum and hence into every metric.
#include "fc_internal.h"

#include <algorithm>

namespace {

// ---------------------------------------------------------------- validation
__global__ void k_validate(const float* __restrict__ x, long long count, FcCtrl* ctrl) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long stride = (long long)gridDim.x * blockDim.x;
    int bad = 0;
    for (; i < count; i += stride) {
        float v = x[i];
        bad |= !isfinite(v);
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&ctrl->bad, 1);
}

// Several sessions' trials: blockIdx.y = session, its blocks stride over its samples.
__global__ void k_validate_batch(PreBatch b) {
    const int s = blockIdx.y;
    const long long count = b.val_prefix[s + 1] - b.val_prefix[s];
    const float* x = b.sp[s].x;
    int bad = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x)
        bad |= !isfinite(x[i]);
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&b.sp[s].ctrl->bad, 1);
}

// ---------------------------------------------------------------- spectrum
// CTA: 32 nodes x 32 bins of one trial. Thread (ty, tx): node ty, bins 4tx..4tx+3.
constexpr int SP_NODES = 32;
constexpr int SP_BINS = 32;
constexpr int SP_CHUNK = 64;

// One CTA's tile (node block bx, bin block by, trial write_from + bz); CTA-uniform exits.
__device__ __forceinline__ void spectrum_tile(const SpectrumArgs& a, int bx, int by, int bz) {
    if (a.ctrl->bad) return;
    const int trial = a.write_from + bz;
    const int node0 = bx * SP_NODES;
    const int bin0 = by * SP_BINS;
    const int tid = threadIdx.x;
    const int ty = tid >> 3, tx = tid & 7;
    __shared__ float xs[SP_NODES][SP_CHUNK + 1];
    __shared__ float2 ws[SP_CHUNK][SP_BINS];

    const float* xt = a.x + (size_t)trial * a.n * a.N;
    float2 acc[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] = make_float2(0.f, 0.f);

    for (int t0 = 0; t0 < a.N; t0 += SP_CHUNK) {
        // stage x[node0..+32][t0..+64] and twiddle[t0..+64][bin0..+32]
        for (int e = tid; e < SP_NODES * SP_CHUNK; e += 256) {
            int r = e / SP_CHUNK, c = e % SP_CHUNK;
            int node = node0 + r, t = t0 + c;
            xs[r][c] = (node < a.n && t < a.N) ? xt[(size_t)node * a.N + t] : 0.f;
        }
        for (int e = tid; e < SP_CHUNK * SP_BINS; e += 256) {
            int r = e / SP_BINS, c = e % SP_BINS;
            int t = t0 + r, b = bin0 + c;
            ws[r][c] = (t < a.N && b < a.B) ? a.twiddle[(size_t)t * a.B + b] : make_float2(0.f, 0.f);
        }
        __syncthreads();
        float2 part[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) part[q] = make_float2(0.f, 0.f);
#pragma unroll 8
        for (int s = 0; s < SP_CHUNK; ++s) {
            float xv = xs[ty][s];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                float2 w = ws[s][tx * 4 + q];
                part[q].x = __fmaf_rn(xv, w.x, part[q].x);
                part[q].y = __fmaf_rn(xv, w.y, part[q].y);
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            acc[q].x = __fadd_rn(acc[q].x, part[q].x);
            acc[q].y = __fadd_rn(acc[q].y, part[q].y);
        }
        __syncthreads();
    }
    const int node = node0 + ty;
    if (node >= a.n) return;
    float scale = a.direct ? 1.f : a.ctrl->scale;
    if (scale == 0.f) scale = 1.f;
    const int slot = a.direct ? bz : (int)((a.ctrl->pushed + trial) % a.slots);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        int b = bin0 + tx * 4 + q;
        if (b < a.B) {
            float2 v = make_float2(__fmul_rn(acc[q].x, scale), __fmul_rn(acc[q].y, scale));
            a.ring[((size_t)slot * a.B + b) * a.n + node] = v;
        }
    }
}

__global__ void __launch_bounds__(256) k_spectrum(SpectrumArgs a) {
    spectrum_tile(a, blockIdx.x, blockIdx.y, blockIdx.z);
}

// One trial of each of several sessions: the sessions' CTAs follow each other
// (spec_prefix), each CTA computes the same tile as k_spectrum would.
__global__ void __launch_bounds__(256) k_spectrum_batch(PreBatch b) {
    const int cta = blockIdx.x;
    int s = 0;
    while (s + 1 < b.nsess && cta >= b.spec_prefix[s + 1]) ++s;
    const SpectrumArgs& a = b.sp[s];
    const int l = cta - b.spec_prefix[s];
    const int gx = (a.n + SP_NODES - 1) / SP_NODES;
    spectrum_tile(a, l % gx, l / gx, 0);
}

// ---------------------------------------------------------------- calibration
// One-time power-of-two prescale: after the first accepted spectra the largest
// |re|, |im| is brought into [1, 2). Every metric is a ratio invariant to a common
// positive factor, and a power of two is exact in FP32, so the metrics are unchanged
// while the squared terms (Im^2, |X|^2) stay far from FP32 underflow for inputs in
// physical units (tesla, volt).
__device__ __forceinline__ float scale_from_bits(unsigned int bits) {
    float m = __uint_as_float(bits);
    if (!(m > 0.f) || !isfinite(m)) return 1.f;
    int e;
    frexpf(m, &e);           // m = f * 2^e, f in [0.5, 1)
    return ldexpf(1.f, 1 - e);  // m * 2^(1-e) in [1, 2)
}

__global__ void k_calibrate(SpectrumArgs a, int phase) {
    FcCtrl* c = a.ctrl;
    if (c->bad || c->scale != 0.f) return;
    const int ntr = a.count - a.write_from;
    const long long per = (long long)a.B * a.n;
    if (phase == 2) {
        if (blockIdx.x == 0 && threadIdx.x == 0) c->scale = scale_from_bits(c->max_bits);
        return;
    }
    const float s = (phase == 1) ? scale_from_bits(c->max_bits) : 1.f;
    unsigned int mloc = 0;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < per * ntr;
         e += (long long)gridDim.x * blockDim.x) {
        long long tr = e / per, off = e % per;
        long long g = c->pushed + a.write_from + tr;
        float2* p = a.ring + (size_t)(g % a.slots) * per + off;
        if (phase == 0) {
            float2 v = *p;
            mloc = max(mloc, __float_as_uint(fmaxf(fabsf(v.x), fabsf(v.y))));
        } else {
            float2 v = *p;
            *p = make_float2(__fmul_rn(v.x, s), __fmul_rn(v.y, s));
        }
    }
    if (phase == 0) {
        for (int o = 16; o > 0; o >>= 1) mloc = max(mloc, __shfl_xor_sync(0xffffffffu, mloc, o));
        if ((threadIdx.x & 31) == 0 && mloc) atomicMax(&c->max_bits, mloc);
    }
}

__device__ __forceinline__ void commit(FcCtrl* c, int count) {
    if (c->bad) {
        c->rejected += count;
        c->bad_latched = 1;
        c->bad = 0;
    } else {
        c->pushed += count;
    }
}

__global__ void k_commit(CommitArgs a) { commit(a.ctrl, a.count); }

// One-trial commits of several sessions; each control block is then copied to the
// session's host snapshot (prescale and rejection count for the host).
__global__ void k_commit_batch(CommitBatch b) {
    const int s = threadIdx.x;
    if (s >= b.nsess) return;
    FcCtrl* c = b.ctrl[s];
    commit(c, 1);
    if (b.snap[s]) *b.snap[s] = *c;
}

}  // namespace

cudaError_t launch_validate(const float* x, long long count, FcCtrl* ctrl, cudaStream_t st) {
    long long blocks = (count + 255) / 256;
    const long long cap = 16LL * fc_device_sms();
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    k_validate<<<(unsigned)blocks, 256, 0, st>>>(x, count, ctrl);
    return cudaGetLastError();
}

cudaError_t launch_spectrum(const SpectrumArgs& a, cudaStream_t st) {
    int ntr = a.count - a.write_from;
    if (ntr <= 0) return cudaSuccess;
    dim3 grid((a.n + SP_NODES - 1) / SP_NODES, (a.B + SP_BINS - 1) / SP_BINS, ntr);
    k_spectrum<<<grid, 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_calibrate(const SpectrumArgs& a, cudaStream_t st, int phase) {
    long long work = (long long)(a.count - a.write_from) * a.B * a.n;
    long long blocks = phase == 2 ? 1 : (work + 255) / 256;
    const long long cap = 8LL * fc_device_sms();
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    k_calibrate<<<(unsigned)blocks, 256, 0, st>>>(a, phase);
    return cudaGetLastError();
}

cudaError_t launch_validate_batch(const PreBatch& b, cudaStream_t st) {
    if (b.nsess <= 0) return cudaSuccess;
    long long most = 0;
    for (int s = 0; s < b.nsess; ++s) most = std::max(most, b.val_prefix[s + 1] - b.val_prefix[s]);
    long long blocks = (most + 255) / 256;
    blocks = std::min(blocks, std::max(1LL, 16LL * fc_device_sms() / b.nsess));
    if (blocks < 1) blocks = 1;
    k_validate_batch<<<dim3((unsigned)blocks, b.nsess), 256, 0, st>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_spectrum_batch(const PreBatch& b, cudaStream_t st) {
    const int ctas = b.nsess > 0 ? b.spec_prefix[b.nsess] : 0;
    if (ctas <= 0) return cudaSuccess;
    k_spectrum_batch<<<ctas, 256, 0, st>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_commit_batch(const CommitBatch& b, cudaStream_t st) {
    if (b.nsess <= 0) return cudaSuccess;
    k_commit_batch<<<1, 32, 0, st>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_commit(const CommitArgs& a, cudaStream_t st) {
    k_commit<<<1, 1, 0, st>>>(a);
    return cudaGetLastError();
}
