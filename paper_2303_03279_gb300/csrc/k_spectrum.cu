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
//
// Wide bands (and any band, where it is cheaper) take the real-FFT method instead when nfft/2
// has no prime factor above 7: one warp per (trial, node) transforms the tapered trial,
// zero-padded to nfft, as the complex sequence z[m] = y[2m] + i y[2m+1] of M = nfft/2 points
// (mixed-radix 4/2/3/5/7 Stockham passes between two shared-memory buffers), and takes only the
// band bins from the even/odd split X[k] = E[k] + e^{-2 pi i k / nfft} O[k] with
// E[k] = (Z[k] + conj Z[M-k]) / 2 and O[k] = (Z[k] - conj Z[M-k]) / 2i. Its FP32 rounding grows
// with the number of passes instead of N.
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

// ---------------------------------------------------------------- real FFT
__device__ __forceinline__ float2 f_cmul(float2 a, float2 b) {
    return make_float2(__fmaf_rn(a.x, b.x, -__fmul_rn(a.y, b.y)), __fmaf_rn(a.x, b.y, __fmul_rn(a.y, b.x)));
}
__device__ __forceinline__ float2 f_add(float2 a, float2 b) { return make_float2(__fadd_rn(a.x, b.x), __fadd_rn(a.y, b.y)); }
__device__ __forceinline__ float2 f_sub(float2 a, float2 b) { return make_float2(__fsub_rn(a.x, b.x), __fsub_rn(a.y, b.y)); }
// -i z and +i z
__device__ __forceinline__ float2 f_mi(float2 z) { return make_float2(z.y, -z.x); }
__device__ __forceinline__ float2 f_pi(float2 z) { return make_float2(-z.y, z.x); }

// e^{-2 pi i k / (2 M)} for 0 <= k < 2 M from the table of its first M values
__device__ __forceinline__ float2 tw_at(const float2* __restrict__ tw, int k, int M) {
    const float2 w = tw[k < M ? k : k - M];
    return k < M ? w : make_float2(-w.x, -w.y);
}

// One Stockham autosort pass of radix R over M points (Govindaraju et al., SC 2008: the
// output of every pass is in natural order, so no bit reversal): for j < M / R, the R inputs
// in[j + r M / R] are twiddled by e^{-2 pi i (j mod Ns) r / (Ns R)}, transformed by an R-point
// DFT and stored at out[(j / Ns) Ns R + (j mod Ns) + s Ns]. Ns = product of the radices of the
// earlier passes.
template <int R>
__device__ __forceinline__ void stockham_pass(const float2* in, float2* out, int M, int Ns,
                                              const float2* __restrict__ tw, int lane) {
    const int nj = M / R;
    const int tstep = 2 * M / (Ns * R), wstep = 2 * M / R;
    for (int j = lane; j < nj; j += 32) {
        const int k = j % Ns;
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = in[j + r * nj];
        if (k != 0) {
#pragma unroll
            for (int r = 1; r < R; ++r) v[r] = f_cmul(v[r], tw_at(tw, k * r * tstep, M));
        }
        float2 V[R];
        if (R == 2) {
            V[0] = f_add(v[0], v[1]);
            V[1] = f_sub(v[0], v[1]);
        } else if (R == 4) {
            const float2 s02 = f_add(v[0], v[2]), d02 = f_sub(v[0], v[2]);
            const float2 s13 = f_add(v[1], v[3]), d13 = f_mi(f_sub(v[1], v[3]));  // -i (v1 - v3)
            V[0] = f_add(s02, s13);
            V[1] = f_add(d02, d13);
            V[2] = f_sub(s02, s13);
            V[3] = f_sub(d02, d13);
        } else {  // R = 3, 5, 7: the R-point DFT by its definition, roots from the table
#pragma unroll
            for (int q = 0; q < R; ++q) {
                float2 acc = v[0];
#pragma unroll
                for (int r = 1; r < R; ++r) acc = f_add(acc, f_cmul(v[r], tw_at(tw, ((r * q) % R) * wstep, M)));
                V[q] = acc;
            }
        }
        const int d = (j / Ns) * Ns * R + k;
#pragma unroll
        for (int q = 0; q < R; ++q) out[d + q * Ns] = V[q];
    }
}

// Warps of a CTA for a transform of M complex points (two buffers of M float2 per warp).
__host__ __device__ __forceinline__ int fft_warps(int M) {
    const int w = 65536 / (M * 16);
    return w < 1 ? 1 : (w > 8 ? 8 : w);
}

__global__ void __launch_bounds__(256) k_spectrum_fft(SpectrumArgs a) {
    if (a.ctrl->bad) return;
    extern __shared__ float2 fbuf[];
    const int M = a.nfft >> 1;
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long item = (long long)blockIdx.x * (blockDim.x >> 5) + wib;
    const int ntr = a.count - a.write_from;
    if (item >= (long long)ntr * a.n) return;  // whole warps: only __syncwarp below
    float2* cur = fbuf + (size_t)wib * 2 * M;
    float2* nxt = cur + M;
    const int tr = (int)(item / a.n), node = (int)(item % a.n);
    const float* x = a.x + ((size_t)(a.write_from + tr) * a.n + node) * a.N;
    // z[m] = y[2m] + i y[2m + 1], y the tapered trial zero-padded to nfft
    for (int m = lane; m < M; m += 32) {
        const int t0 = 2 * m, t1 = t0 + 1;
        const float v0 = t0 < a.N ? __fmul_rn(x[t0], a.taper[t0]) : 0.f;
        const float v1 = t1 < a.N ? __fmul_rn(x[t1], a.taper[t1]) : 0.f;
        cur[m] = make_float2(v0, v1);
    }
    __syncwarp();
    int Ns = 1;
    for (int st = 0; st < a.fft_stages; ++st) {
        const int R = (int)((a.fft_radices >> (4 * st)) & 15u);
        if (R == 4) stockham_pass<4>(cur, nxt, M, Ns, a.fft_tw, lane);
        else if (R == 2) stockham_pass<2>(cur, nxt, M, Ns, a.fft_tw, lane);
        else if (R == 3) stockham_pass<3>(cur, nxt, M, Ns, a.fft_tw, lane);
        else if (R == 5) stockham_pass<5>(cur, nxt, M, Ns, a.fft_tw, lane);
        else stockham_pass<7>(cur, nxt, M, Ns, a.fft_tw, lane);
        __syncwarp();
        float2* t = cur;
        cur = nxt;
        nxt = t;
        Ns *= R;
    }
    float scale = a.direct ? 1.f : a.ctrl->scale;
    if (scale == 0.f) scale = 1.f;
    const int slot = a.direct ? tr : (int)((a.ctrl->pushed + a.write_from + tr) % a.slots);
    float2* out = a.ring + (size_t)slot * a.B * a.n + node;
    for (int b = lane; b < a.B; b += 32) {
        const int k = a.first_bin + b;  // 0 <= k <= M
        const float2 zk = cur[k == M ? 0 : k];
        const float2 zm = cur[k == 0 ? 0 : M - k];
        const float2 e = make_float2(0.5f * __fadd_rn(zk.x, zm.x), 0.5f * __fsub_rn(zk.y, zm.y));
        const float2 o = make_float2(0.5f * __fadd_rn(zk.y, zm.y), -0.5f * __fsub_rn(zk.x, zm.x));
        const float2 w = k < M ? a.fft_tw[k] : make_float2(-1.f, 0.f);
        const float2 wo = f_cmul(w, o);
        out[(size_t)b * a.n] = make_float2(__fmul_rn(__fadd_rn(e.x, wo.x), scale), __fmul_rn(__fadd_rn(e.y, wo.y), scale));
    }
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
    if (a.fft) {
        const int M = a.nfft / 2, wpb = fft_warps(M);
        const int smem = wpb * 2 * M * (int)sizeof(float2);
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(k_spectrum_fft, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            if (e != cudaSuccess) return e;
        }
        const long long items = (long long)ntr * a.n;
        k_spectrum_fft<<<(unsigned)((items + wpb - 1) / wpb), 32 * wpb, smem, st>>>(a);
        return cudaGetLastError();
    }
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
    for (int s = 0; s < b.nsess; ++s)  // sessions on the FFT method: a launch each
        if (b.sp[s].fft) {
            cudaError_t e = launch_spectrum(b.sp[s], st);
            if (e != cudaSuccess) return e;
        }
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
