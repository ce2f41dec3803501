// fc_noalloc.cu - spectral networks of one window without any device allocation.
//
// Some callers cannot call cudaMalloc: a real-time acquisition loop where an allocation
// (which may synchronize the whole device and take an unbounded time) would break the
// per-trial deadline, or a host application whose device memory is owned entirely by
// another allocator (a framework's caching allocator, a pre-reserved pool). For them,
// fc_window_networks_noalloc computes the band-averaged spectral networks of a window
// from spectra the caller already holds on the device, into an output the caller owns,
// and keeps every intermediate (window control block, per-node PSD sums, tile tables,
// band partial sums) in one file-scope device array of FC_NOALLOC_SCRATCH_BYTES that
// the library holds on every GPU that loads it, until the process exits. Like a session,
// it brings the spectra into a fixed range by an exact power-of-two factor applied as the
// kernels read them.
#include <algorithm>
#include <cstdint>
#include <mutex>

#include "fc_internal.h"

namespace {

constexpr size_t kScratchBytes = (size_t)FC_NOALLOC_SCRATCH_BYTES;

// The shared scratch: every call uses it, and it keeps the last call's contents.
static __device__ __align__(256) unsigned char fc_noalloc_scratch[kScratchBytes];

// Device address of the scratch array and multiprocessor count, per device (the host-side
// symbol is only a stand-in). Only a successful lookup is kept: a failed one (a sticky error
// from earlier work, a call made during stream capture) is tried again by the next call.
constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_addr[kMaxDevices];
int g_scratch_sms[kMaxDevices];

cudaError_t scratch_address(int dev, void** out, int* sms) {
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, fc_noalloc_scratch);
        if (e != cudaSuccess || !p) return e != cudaSuccess ? e : cudaErrorInvalidSymbol;
        g_scratch_addr[dev] = p;
        g_scratch_sms[dev] = fc_device_sms(dev);
    }
    *out = g_scratch_addr[dev];
    *sms = g_scratch_sms[dev];
    return cudaSuccess;
}

// Power-of-two prescale of the caller's spectra, as a session applies to its own: the largest
// |re|, |im| of the window is brought into [1, 2) so that the squared terms (Im^2, |X|^2)
// stay far from FP32 underflow for spectra in physical units. A power of two is exact and
// every metric is invariant to a common positive factor. The kernels apply it as they read
// the spectra (FcCtrl::in_scale); the caller's buffer is not written.
__global__ void k_noalloc_max(const float* __restrict__ v, long long count, FcCtrl* ctrl) {
    unsigned int m = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x) {
        const float x = fabsf(v[i]);
        if (x <= 3.4028234663852886e38f) m = max(m, __float_as_uint(x));  // finite values only
    }
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m) atomicMax(&ctrl->max_bits, m);
}

__global__ void k_noalloc_scale(FcCtrl* ctrl) {
    const float m = __uint_as_float(ctrl->max_bits);
    float s = 1.f;
    if (m > 0.f) {
        int e;
        frexpf(m, &e);          // m = f 2^e, f in [0.5, 1)
        s = ldexpf(1.f, 1 - e); // m s in [1, 2)
    }
    ctrl->in_scale = s;
}

__global__ void k_noalloc_tiles(unsigned short* ta, unsigned short* tb, int nt) {
    const int tp = blockIdx.x * blockDim.x + threadIdx.x;
    if (tp >= nt * (nt + 1) / 2) return;
    int r = tp, a = 0;
    while (r >= nt - a) {
        r -= nt - a;
        ++a;
    }
    ta[tp] = (unsigned short)a;
    tb[tp] = (unsigned short)(a + r);
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

fc_status noalloc_fail(fc_status st, const char* msg) {
    fc_internal_set_error(msg);
    return st;
}

}  // namespace

extern "C" fc_status fc_window_networks_noalloc(const float* spectra, int n_trials, int n_bins, int n_nodes,
                                                uint32_t metric_mask, float* out, size_t out_len,
                                                void* stream) {
    if (!spectra || !out) return noalloc_fail(FC_ERR_INVALID_ARG, "spectra and out must be device pointers");
    if (n_trials < 1 || n_bins < 1 || n_nodes < 2 || n_nodes > 65535 * FC_T)
        return noalloc_fail(FC_ERR_INVALID_ARG, "need n_trials >= 1, n_bins >= 1, n_nodes >= 2");
    if ((metric_mask & ~(uint32_t)FC_SPECTRAL_METRICS) || !(metric_mask & FC_SPECTRAL_METRICS))
        return noalloc_fail(FC_ERR_INVALID_ARG, "metric_mask must be a nonzero subset of the spectral metrics");
    const long long P = (long long)n_nodes * (n_nodes - 1) / 2;
    if (out_len < (size_t)(7 * P)) return noalloc_fail(FC_ERR_INVALID_ARG, "out_len must be >= 7 * n(n-1)/2");

    // scratch plan: control block | PSD sums (double) | 1/sqrt(PSD) | tile tables | band partials
    const int nt = (n_nodes + FC_T - 1) / FC_T;
    const int ntp = nt * (nt + 1) / 2;
    const size_t off_psd = align256(sizeof(FcCtrl));
    const size_t off_inv = align256(off_psd + sizeof(double) * (size_t)n_bins * n_nodes);
    const size_t off_ta = align256(off_inv + sizeof(float) * (size_t)n_bins * n_nodes);
    const size_t off_tb = align256(off_ta + sizeof(unsigned short) * (size_t)ntp);
    const size_t off_part = align256(off_tb + sizeof(unsigned short) * (size_t)ntp);
    if (off_part > kScratchBytes)
        return noalloc_fail(FC_ERR_INVALID_ARG,
                            "window too large for the fixed scratch (n_bins * n_nodes must stay below ~1.3 M)");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    void* base = nullptr;
    if (e == cudaSuccess) e = scratch_address(dev, &base, &sms);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return noalloc_fail(FC_ERR_CUDA, cudaGetErrorString(e));
    }
    // bin groups: as many as fill the GPU (two CTAs per SM, twice over) and fit in the
    // remaining scratch
    int groups = std::min(n_bins, std::max(1, (sms * 4 + ntp - 1) / ntp));
    const size_t per_group = sizeof(float) * 7 * (size_t)P;
    while (groups > 1 && off_part + per_group * groups > kScratchBytes) --groups;
    const int group_bins = (n_bins + groups - 1) / groups;
    groups = (n_bins + group_bins - 1) / group_bins;
    unsigned char* s = static_cast<unsigned char*>(base);
    FcCtrl* ctrl = reinterpret_cast<FcCtrl*>(s);
    double* psd = reinterpret_cast<double*>(s + off_psd);
    float* inv = reinterpret_cast<float*>(s + off_inv);
    unsigned short* ta = reinterpret_cast<unsigned short*>(s + off_ta);
    unsigned short* tb = reinterpret_cast<unsigned short*>(s + off_tb);
    float* partial = groups > 1 ? reinterpret_cast<float*>(s + off_part) : nullptr;
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    // the window control block must start at zero: trials [0, n_trials) of the given spectra
    e = cudaMemsetAsync(ctrl, 0, sizeof(FcCtrl), st);
    if (e == cudaSuccess) {
        k_noalloc_tiles<<<(ntp + 255) / 256, 256, 0, st>>>(ta, tb, nt);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        const long long count = 2LL * n_trials * n_bins * n_nodes;
        const long long blocks = std::min<long long>((count + 255) / 256, 8LL * sms);
        k_noalloc_max<<<(unsigned)std::max(1LL, blocks), 256, 0, st>>>(spectra, count, ctrl);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        k_noalloc_scale<<<1, 1, 0, st>>>(ctrl);
        e = cudaGetLastError();
    }
    const float2* ring = reinterpret_cast<const float2*>(spectra);
    if (e == cudaSuccess) {
        NodeArgs na{ring, psd, inv, n_trials, n_nodes, n_bins, n_trials, 1, ctrl, n_trials};
        e = launch_node(na, st);
    }
    PairArgs pa{};
    pa.ring = ring;
    pa.inv_psd = inv;
    pa.acc = nullptr;
    pa.tile_a = ta;
    pa.tile_b = tb;
    pa.net_spec = out;  // the seven spectral planes, COH .. DSWPLI
    pa.partial = partial;
    pa.slots = n_trials;
    pa.n = n_nodes;
    pa.B = n_bins;
    pa.fsel0 = 0;
    pa.fsel1 = n_bins;
    pa.W = n_trials;
    pa.ntp = ntp;
    pa.P = P;
    pa.groups = groups;
    pa.group_bins = group_bins;
    pa.mask = metric_mask;
    pa.finalize = 1;
    pa.update = 1;
    pa.write_acc = 0;
    pa.count = n_trials;
    pa.grid_ctas = 2 * sms;
    pa.ctrl = ctrl;
    if (e == cudaSuccess) e = launch_window_sums(pa, st);
    if (e == cudaSuccess && groups > 1) e = launch_band_reduce(pa, st);
    if (e != cudaSuccess) return noalloc_fail(FC_ERR_CUDA, cudaGetErrorString(e));
    return FC_OK;
}
