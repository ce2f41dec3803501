// fc_fir.cu - FIR filtering of the incoming multichannel stream, upstream of the sessions.
//
// Methods 2.4 (Noise Reduction plug-in): FIR low-, high- and band-pass filters are designed
// on the fly from cut-off frequencies, transition bandwidth and number of taps, all with a
// linear phase; data arrive in blocks and overlap-add carries the filter's tail across the
// block boundaries. Here the taps come from the window method (ideal response as a
// difference of sinc low-passes, times a Hamming window, odd length, designed in FP64 on
// the host), and each block is filtered by a direct causal convolution whose state - the
// last T - 1 input samples of every channel - carries over to the next block: the output is
// the filtered continuous stream, the same result overlap-add gives.
//
// CTA: one channel x 256 consecutive outputs; the taps and the input segment
// (state | block) it needs are staged in shared memory; each output is one FMA chain in a
// fixed order, so the result does not depend on the block sizes. C x L x T FMAs per block.
#include <cmath>
#include <cstring>
#include <vector>

#include "fc_internal.h"

namespace {

constexpr int OUT_PER_CTA = 256;
constexpr int MAX_TAPS = 8191;

__global__ void __launch_bounds__(OUT_PER_CTA) k_fir(const float* __restrict__ x, const float* __restrict__ state,
                                                     const float* __restrict__ h, float* __restrict__ y, int L,
                                                     int T) {
    extern __shared__ float sm[];
    float* th = sm;          // [T]
    float* seg = sm + T;     // [OUT_PER_CTA + T - 1]
    const int c = blockIdx.y;
    const int t0 = blockIdx.x * OUT_PER_CTA;
    const float* xc = x + (size_t)c * L;
    const float* sc = state + (size_t)c * (T - 1);
    for (int k = threadIdx.x; k < T; k += blockDim.x) th[k] = h[k];
    // seg[i] = x_ext[t0 + i], x_ext = [state (T - 1) | block (L)]
    const int seg_len = OUT_PER_CTA + T - 1;
    for (int i = threadIdx.x; i < seg_len; i += blockDim.x) {
        const int e = t0 + i;
        float v = 0.f;
        if (e < T - 1)
            v = sc[e];
        else if (e - (T - 1) < L)
            v = xc[e - (T - 1)];
        seg[i] = v;
    }
    __syncthreads();
    const int t = t0 + threadIdx.x;
    if (t >= L) return;
    // y[t] = sum_k h[k] x_ext[t + T - 1 - k]
    float acc = 0.f;
    const float* s = seg + threadIdx.x + T - 1;
    for (int k = 0; k < T; ++k) acc = __fmaf_rn(th[k], s[-k], acc);
    y[(size_t)c * L + t] = acc;
}

// new state = the last T - 1 samples of [state | block]
__global__ void k_fir_state(const float* __restrict__ x, const float* __restrict__ state, float* __restrict__ next,
                            int L, int T, int C) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int S = T - 1;
    if (i >= (long long)C * S) return;
    const int c = (int)(i / S), j = (int)(i % S);
    const long long e = (long long)L + j;  // index into x_ext
    next[i] = e < S ? state[(size_t)c * S + e] : x[(size_t)c * L + (e - S)];
}

double sinc(double v) {
    if (v == 0.0) return 1.0;
    const double pv = 3.14159265358979323846 * v;
    return std::sin(pv) / pv;
}

}  // namespace

struct fc_fir {
    int C = 0, T = 0;
    std::vector<double> taps;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0;
    float* d_h = nullptr;
    float* d_state[2] = {nullptr, nullptr};
    int cur = 0;
    float* d_x = nullptr;  // staging for host blocks [C][cap]
    float* d_y = nullptr;
    int cap = 0;
};

extern "C" {

fc_status fc_fir_create(int n_channels, double fs, fc_fir_kind kind, double f_lo, double f_hi, double transition_hz,
                        int n_taps, void* stream, fc_fir** out) {
    if (!out) {
        fc_internal_set_error("out is NULL");
        return FC_ERR_INVALID_ARG;
    }
    *out = nullptr;
    const double nyq = fs / 2.0;
    bool ok = n_channels >= 1 && n_channels <= 65535 && fs > 0.0 && n_taps >= 0 &&
              (n_taps > 0 || transition_hz > 0.0);
    if (kind == FC_FIR_LOWPASS) ok = ok && f_hi > 0.0 && f_hi < nyq;
    else if (kind == FC_FIR_HIGHPASS) ok = ok && f_lo > 0.0 && f_lo < nyq;
    else if (kind == FC_FIR_BANDPASS) ok = ok && f_lo > 0.0 && f_hi > f_lo && f_hi < nyq;
    else ok = false;
    if (!ok) {
        fc_internal_set_error("bad filter settings (cut-offs inside (0, fs/2), taps or a transition width)");
        return FC_ERR_INVALID_ARG;
    }
    int T = n_taps > 0 ? n_taps : (int)std::ceil(3.3 * fs / transition_hz);
    if (T % 2 == 0) ++T;
    if (T > MAX_TAPS) {
        fc_internal_set_error("more than 8191 taps");
        return FC_ERR_INVALID_ARG;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        fc_internal_set_error("no CUDA device: this library has no CPU path");
        return FC_ERR_CUDA;
    }
    fc_fir* f = new fc_fir();
    f->C = n_channels;
    f->T = T;
    f->taps.resize(T);
    const double m = (T - 1) / 2.0;
    for (int k = 0; k < T; ++k) {
        const double d = k - m;
        auto lowpass = [&](double fc) { return 2.0 * fc / fs * sinc(2.0 * fc / fs * d); };
        double v;
        if (kind == FC_FIR_LOWPASS) v = lowpass(f_hi);
        else if (kind == FC_FIR_HIGHPASS) v = (d == 0.0 ? 1.0 : 0.0) - lowpass(f_lo);
        else v = lowpass(f_hi) - lowpass(f_lo);
        const double w = T > 1 ? 0.54 - 0.46 * std::cos(2.0 * 3.14159265358979323846 * k / (T - 1)) : 1.0;
        f->taps[k] = v * w;
    }
    cudaGetDevice(&f->device);
    f->stream = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
    if (!f->stream) {
        e = cudaStreamCreateWithFlags(&f->stream, cudaStreamNonBlocking);
        f->own_stream = e == cudaSuccess;
    }
    std::vector<float> hf(T);
    for (int k = 0; k < T; ++k) hf[k] = (float)f->taps[k];
    const size_t sb = (size_t)n_channels * (T > 1 ? T - 1 : 1) * sizeof(float);
    if (e == cudaSuccess) e = cudaMalloc(&f->d_h, T * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&f->d_state[0], sb);
    if (e == cudaSuccess) e = cudaMalloc(&f->d_state[1], sb);
    // on the filter's stream (non-blocking: not ordered with the legacy stream), then waited for
    if (e == cudaSuccess) e = cudaMemcpyAsync(f->d_h, hf.data(), T * sizeof(float), cudaMemcpyHostToDevice, f->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(f->d_state[0], 0, sb, f->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(f->d_state[1], 0, sb, f->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(f->stream);
    if (e == cudaSuccess) {  // the attribute is per kernel: set it for the longest filter allowed
        const int smem_max = (int)((2 * MAX_TAPS + OUT_PER_CTA - 1) * sizeof(float));
        e = cudaFuncSetAttribute(k_fir, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max);
    }
    if (e != cudaSuccess) {
        fc_internal_set_error(cudaGetErrorString(e));
        fc_fir_destroy(f);
        return FC_ERR_CUDA;
    }
    *out = f;
    return FC_OK;
}

fc_status fc_fir_get_taps(fc_fir* f, double* taps, int max_taps, int* n_taps) {
    if (!f || !n_taps) {
        fc_internal_set_error("NULL argument");
        return FC_ERR_INVALID_ARG;
    }
    *n_taps = f->T;
    if (taps) {
        if (max_taps < f->T) {
            fc_internal_set_error("taps buffer too small");
            return FC_ERR_INVALID_ARG;
        }
        std::memcpy(taps, f->taps.data(), f->T * sizeof(double));
    }
    return FC_OK;
}

fc_status fc_fir_process(fc_fir* f, const float* x, float* y, int block_len, int on_device) {
    if (!f || !x || !y || block_len < 1) {
        fc_internal_set_error("NULL argument or empty block");
        return FC_ERR_INVALID_ARG;
    }
    cudaSetDevice(f->device);
    const size_t bytes = (size_t)f->C * block_len * sizeof(float);
    const float* dx = x;
    float* dy = y;
    cudaError_t e = cudaSuccess;
    if (!on_device) {
        if (f->cap < block_len) {
            cudaFree(f->d_x);
            cudaFree(f->d_y);
            f->d_x = f->d_y = nullptr;
            f->cap = 0;
            e = cudaMalloc(&f->d_x, bytes);
            if (e == cudaSuccess) e = cudaMalloc(&f->d_y, bytes);
            if (e == cudaSuccess) f->cap = block_len;
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(f->d_x, x, bytes, cudaMemcpyHostToDevice, f->stream);
        dx = f->d_x;
        dy = f->d_y;
    }
    if (e == cudaSuccess) {
        dim3 grid((block_len + OUT_PER_CTA - 1) / OUT_PER_CTA, f->C);
        const int smem = (int)((f->T + OUT_PER_CTA + f->T - 1) * sizeof(float));
        k_fir<<<grid, OUT_PER_CTA, smem, f->stream>>>(dx, f->d_state[f->cur], f->d_h, dy, block_len, f->T);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && f->T > 1) {
        const long long n = (long long)f->C * (f->T - 1);
        k_fir_state<<<(unsigned)((n + 255) / 256), 256, 0, f->stream>>>(dx, f->d_state[f->cur], f->d_state[f->cur ^ 1],
                                                                       block_len, f->T, f->C);
        e = cudaGetLastError();
        f->cur ^= 1;
    }
    if (e == cudaSuccess && !on_device) {
        e = cudaMemcpyAsync(y, dy, bytes, cudaMemcpyDeviceToHost, f->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(f->stream);
    }
    if (e != cudaSuccess) {
        fc_internal_set_error(cudaGetErrorString(e));
        return FC_ERR_CUDA;
    }
    return FC_OK;
}

fc_status fc_fir_reset(fc_fir* f) {
    if (!f) {
        fc_internal_set_error("NULL filter");
        return FC_ERR_INVALID_ARG;
    }
    cudaSetDevice(f->device);
    const size_t sb = (size_t)f->C * (f->T > 1 ? f->T - 1 : 1) * sizeof(float);
    cudaError_t e = cudaMemsetAsync(f->d_state[f->cur], 0, sb, f->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(f->stream);
    if (e != cudaSuccess) {
        fc_internal_set_error(cudaGetErrorString(e));
        return FC_ERR_CUDA;
    }
    return FC_OK;
}

fc_status fc_fir_destroy(fc_fir* f) {
    if (!f) return FC_OK;
    cudaSetDevice(f->device);
    if (f->stream) cudaStreamSynchronize(f->stream);
    cudaFree(f->d_h);
    cudaFree(f->d_state[0]);
    cudaFree(f->d_state[1]);
    cudaFree(f->d_x);
    cudaFree(f->d_y);
    if (f->own_stream) cudaStreamDestroy(f->stream);
    delete f;
    return FC_OK;
}

}  // extern "C"
