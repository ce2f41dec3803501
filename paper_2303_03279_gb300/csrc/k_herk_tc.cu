// k_herk_tc.cu - full-window linear pair sums on the 5th-generation tensor cores
// (tcgen05.mma, accumulators in TMEM, operands staged by TMA bulk copies).
//
// Per bin f, the linear sums over the K trials of the window are Hermitian rank-K
// products (Methods 2.4: running sums of CSD; Supplementary Information 1: COHY, PLV):
//   S_csd(i, j) = sum_k X_ki X_kj*,   S_u(i, j) = sum_k u_ki u_kj*   (u = X/|X|).
// With A_r = [Re X | Im X] and A_i = [Im X | -Re X] (rows = nodes, inner = 2K trials):
//   Re S_csd = A_r(rows i) A_r(rows j)^T,   Im S_csd = A_i(rows i) A_r(rows j)^T,
// and the same with U for the phasor sums: four real GEMMs of 128 x 128 x 2K per
// (128-node tile pair, bin), kind::f16 (BF16 or FP16 operands) or kind::tf32, FP32
// accumulation. COH, IMAGCOHY and PLV of the bin are finalized from TMEM and written per
// bin; the band average follows in a small reduction kernel. The non-linear sums
// (signs, |Im|, Im^2) cannot be contracted and run on the CUDA cores (k_nonlin).
//
// Operand layout (built by k_pack_operands from the ring of FP32 spectra): for each
// (tile, bin, operand kind, 128-byte K-chunk) one contiguous 16 KB block in the
// K-major, no-swizzle canonical layout of core matrices (8 rows x 16 bytes):
//   byte offset = ((m / 8) * 8 + kc) * 128 + (m % 8) * 16 + (byte within the 16-byte row chunk)
// i.e. leading (K-direction) core-matrix stride 128 B, stride (M/N-direction) 1024 B.
// One cp.async.bulk moves a block into shared memory as is.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "fc_internal.h"
#include "mbar.cuh"

namespace {

using namespace fcmbar;

constexpr int TILE = 128;             // nodes per tile (M = N = 128)
constexpr int CHUNK_BYTES = 16384;     // 128 rows x 128 bytes of K
constexpr int NOPS = 6;                // XR(a), XI(a), UR(a), UI(a), XR(b), UR(b)
constexpr int STAGE_BYTES = NOPS * CHUNK_BYTES;
constexpr int SMEM_BYTES = 2 * STAGE_BYTES + 128;  // + barriers and the TMEM address
constexpr uint32_t TMEM_COLS = 512;    // 4 accumulators x 128 FP32 columns

// Shared-memory matrix descriptor: K-major, no swizzle; LBO = 128 B (next core matrix
// along K), SBO = 1024 B (next 8-row group), descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((128u >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((1024u >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor: D = F32, A/B format (F16 = 0, BF16 = 1, TF32 = 2), both K-major,
// N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t make_idesc(uint32_t ab_format, uint32_t M, uint32_t N) {
    return (1u << 4) | (ab_format << 7) | (ab_format << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

template <int KIND>  // 0 = kind::f16 (BF16/FP16 operands), 1 = kind::tf32
__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
    if (KIND == 0)
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
            "l"(da), "l"(db), "r"(idesc), "r"(acc));
    else
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
            "l"(da), "l"(db), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}

__device__ __forceinline__ long long packed_index(int i, int j, int n) {
    return (long long)i * n - (long long)i * (i + 1) / 2 + (j - i - 1);
}

__device__ __forceinline__ const unsigned char* op_block(const HerkArgs& a, int tile, int f, int kind, int chunk) {
    return a.ops + ((((size_t)tile * a.B + f) * 4 + kind) * a.nchunks + chunk) * (size_t)CHUNK_BYTES;
}

template <int KIND>
__global__ void __launch_bounds__(128, 1) k_herk_tc(HerkArgs a) {
    extern __shared__ __align__(1024) unsigned char smem[];
    FcCtrl* c = const_cast<FcCtrl*>(a.ctrl);
    if (c->bad) return;
    const int units = a.ntp * a.B;
    if ((int)blockIdx.x >= units) return;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + 2 * STAGE_BYTES);  // [2]
    uint64_t* freeb = full + 2;                                            // [2]
    uint64_t* accb = full + 4;                                             // [1]
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(full + 6);
    const int tid = threadIdx.x, warp = tid >> 5;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(&full[0], 1);
        mbar_init(&full[1], 1);
        mbar_init(&freeb[0], 1);
        mbar_init(&freeb[1], 1);
        mbar_init(accb, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t idesc = make_idesc(KIND == 1 ? 2u : (a.ab_format == 1 ? 1u : 0u), TILE, TILE);
    const long long wend = c->pushed + a.count;
    const int K = (int)(wend - ((a.W > 0 && wend > a.W) ? wend - a.W : 0));
    const float inv_K = 1.0f / (float)K;

    uint32_t full_phase[2] = {0, 0}, free_phase[2] = {0, 0}, acc_phase = 0;
    int loads = 0;       // chunk loads issued (stage = loads % 2); load s = chunk s of this CTA's sequence
    int consumed = 0;    // chunks consumed by MMAs
    bool failed = false;
    const long long seq_len = (long long)((units - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x) * a.nchunks;

    // the CTA's chunk sequence: position s -> unit blockIdx.x + (s / nchunks) * gridDim.x, chunk s % nchunks
    auto issue_next_load = [&]() {  // thread 0 only
        if (loads >= seq_len) return;
        const int u = (int)blockIdx.x + (loads / a.nchunks) * (int)gridDim.x;
        const int ch = loads % a.nchunks;
        const int tp = u / a.B, f = u % a.B;
        const int ta = a.tile_a[tp], tb = a.tile_b[tp];
        const int st = loads & 1;
        if (loads >= 2) {  // the stage's previous MMAs must be done reading it
            if (!mbar_wait_bounded(&freeb[st], free_phase[st])) failed = true;
            free_phase[st] ^= 1;
        }
        unsigned char* dst = smem + st * STAGE_BYTES;
        mbar_expect_tx(&full[st], STAGE_BYTES);
        bulk_g2s(dst + 0 * CHUNK_BYTES, op_block(a, ta, f, 0, ch), CHUNK_BYTES, &full[st]);
        bulk_g2s(dst + 1 * CHUNK_BYTES, op_block(a, ta, f, 1, ch), CHUNK_BYTES, &full[st]);
        bulk_g2s(dst + 2 * CHUNK_BYTES, op_block(a, ta, f, 2, ch), CHUNK_BYTES, &full[st]);
        bulk_g2s(dst + 3 * CHUNK_BYTES, op_block(a, ta, f, 3, ch), CHUNK_BYTES, &full[st]);
        bulk_g2s(dst + 4 * CHUNK_BYTES, op_block(a, tb, f, 0, ch), CHUNK_BYTES, &full[st]);
        bulk_g2s(dst + 5 * CHUNK_BYTES, op_block(a, tb, f, 2, ch), CHUNK_BYTES, &full[st]);
        ++loads;
    };

    int u = blockIdx.x;
    if (tid == 0) {
        issue_next_load();
        issue_next_load();
    }
    while (u < units) {
        const int tp = u / a.B, f = u % a.B;
        const int ta = a.tile_a[tp], tb = a.tile_b[tp];
        const int nu = u + (int)gridDim.x;
        if (tid == 0) {
            for (int ch = 0; ch < a.nchunks; ++ch) {
                const int st = consumed & 1;
                if (!mbar_wait_bounded(&full[st], full_phase[st])) failed = true;
                full_phase[st] ^= 1;
                fence_after();
                const uint32_t base = smem_u32(smem + st * STAGE_BYTES);
#pragma unroll
                for (int ks = 0; ks < 4; ++ks) {
                    const uint32_t acc = (ch > 0 || ks > 0) ? 1u : 0u;
                    const uint32_t off = ks * 256;
                    const uint64_t dxr_a = smem_desc(base + 0 * CHUNK_BYTES + off);
                    const uint64_t dxi_a = smem_desc(base + 1 * CHUNK_BYTES + off);
                    const uint64_t dur_a = smem_desc(base + 2 * CHUNK_BYTES + off);
                    const uint64_t dui_a = smem_desc(base + 3 * CHUNK_BYTES + off);
                    const uint64_t dxr_b = smem_desc(base + 4 * CHUNK_BYTES + off);
                    const uint64_t dur_b = smem_desc(base + 5 * CHUNK_BYTES + off);
                    // transposed products: D^T[j][i] (TMEM lane = column node j), so that the
                    // epilogue's warp-wide stores run along j, contiguous in the packed triangle
                    mma<KIND>(tmem + 0 * TILE, dxr_b, dxr_a, idesc, acc);
                    mma<KIND>(tmem + 1 * TILE, dxr_b, dxi_a, idesc, acc);
                    mma<KIND>(tmem + 2 * TILE, dur_b, dur_a, idesc, acc);
                    mma<KIND>(tmem + 3 * TILE, dur_b, dui_a, idesc, acc);
                }
                mma_commit(&freeb[st]);  // the stage may be refilled once these MMAs have read it
                ++consumed;
                issue_next_load();       // keep two chunks in flight along the sequence
            }
            mma_commit(accb);
        }
        // epilogue: thread t owns TMEM lane t = column node j of the tile pair; TMEM columns
        // are the row nodes i
        const bool ok = mbar_wait_bounded(accb, acc_phase);
        acc_phase ^= 1;
        fence_after();
        const int fail_any = __syncthreads_or((!ok || failed) ? 1 : 0);
        if (fail_any) {
            if (tid == 0) atomicOr(&c->timeout, 1);
            break;
        }
        const int j = tb * TILE + tid;
        const float inv_j = j < a.n ? a.inv_psd[(size_t)f * a.n + j] : 0.f;
        const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
        for (int i0 = 0; i0 < TILE; i0 += 16) {
            float cre[16], cim[16], ure[16], uim[16];
            tmem_ld16(lane_base + 0 * TILE + i0, cre);
            tmem_ld16(lane_base + 1 * TILE + i0, cim);
            tmem_ld16(lane_base + 2 * TILE + i0, ure);
            tmem_ld16(lane_base + 3 * TILE + i0, uim);
            if (j >= a.n) continue;
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int i = ta * TILE + i0 + q;
                if (j <= i || i >= a.n) continue;
                const float inv_i = a.inv_psd[(size_t)f * a.n + i];
                const float r = __fmul_rn(__fmul_rn(cre[q], inv_i), inv_j);
                const float m = __fmul_rn(__fmul_rn(cim[q], inv_i), inv_j);
                const long long p = packed_index(i, j, a.n);
                float* out = a.bins_out + (size_t)f * 3 * a.P;
                out[p] = sqrtf(__fmaf_rn(r, r, __fmul_rn(m, m)));
                out[a.P + p] = m;
                out[2 * a.P + p] = __fmul_rn(sqrtf(__fmaf_rn(ure[q], ure[q], __fmul_rn(uim[q], uim[q]))), inv_K);
            }
        }
        fence_before();
        __syncthreads();  // TMEM free for the next unit's MMAs
        fence_after();
        u = nu;
    }
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

// ------------------------------------------------------------------ operand packing
// One thread per 16-byte row chunk of a core matrix: operand kind, tile, bin, node row m,
// 16-byte K unit. Elements k of the 2K inner dimension: k < K -> trial k, first half;
// K <= k < 2K -> trial k - K, second half; beyond 2K -> 0.
//   XR = [Re X | Im X], XI = [Im X | -Re X], UR = [Re u | Im u], UI = [Im u | -Re u]
__device__ __forceinline__ float2 phasor_of_x(float2 X) {
    float m2 = __fmaf_rn(X.x, X.x, __fmul_rn(X.y, X.y));
    float r = (m2 > 0.0f) ? rsqrtf(m2) : 0.0f;
    return make_float2(__fmul_rn(X.x, r), __fmul_rn(X.y, r));
}

__device__ __forceinline__ float op_value(int kind, float2 X, int part) {
    if (kind >= 2) X = phasor_of_x(X);
    if (kind == 0 || kind == 2) return part ? X.y : X.x;
    return part ? -X.x : X.y;
}

__global__ void k_pack_operands(PackArgs a) {
    const FcCtrl* c = a.ctrl;
    if (c->bad) return;
    const long long end = c->pushed + a.count;
    const long long start = (a.W > 0 && end > a.W) ? end - a.W : 0;
    const int K = (int)(end - start);
    const int esize = a.ab_format == 2 ? 4 : 2;
    const int per16 = 16 / esize;                 // elements per 16-byte unit
    const long long units_per_block = (long long)TILE * 8;  // 128 rows x 8 units of 16 bytes
    const long long total = (long long)a.ntiles * a.B * 4 * a.nchunks * units_per_block;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        long long rest = e;
        const int r = (int)(rest % 8); rest /= 8;       // row within core matrix
        const int kc = (int)(rest % 8); rest /= 8;      // core matrix along K within the chunk
        const int m8 = (int)(rest % 16); rest /= 16;    // 8-row group
        const int ch = (int)(rest % a.nchunks); rest /= a.nchunks;
        const int kind = (int)(rest % 4); rest /= 4;
        const int f = (int)(rest % a.B); rest /= a.B;
        const int tile = (int)rest;
        const int m = m8 * 8 + r;
        const int node = tile * TILE + m;
        const int k0 = (ch * 8 + kc) * per16;           // first inner index of this 16-byte unit
        float v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int k = k0 + q;
            float val = 0.f;
            if (q < per16 && node < a.n && k < 2 * K) {
                const int part = k >= K;
                const long long trial = start + (part ? k - K : k);
                const float2 X = a.ring[((size_t)(trial % a.slots) * a.B + f) * a.n + node];
                val = op_value(kind, X, part);
            }
            v[q] = val;
        }
        unsigned char* dst = a.ops + ((((size_t)tile * a.B + f) * 4 + kind) * a.nchunks + ch) * (size_t)CHUNK_BYTES +
                             (size_t)(m8 * 8 + kc) * 128 + r * 16;
        uint4 w;
        if (a.ab_format == 2) {  // TF32: round to nearest (ties away), stored in 32-bit words
            uint32_t t[4];
            for (int q = 0; q < 4; ++q) asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(t[q]) : "f"(v[q]));
            w = make_uint4(t[0], t[1], t[2], t[3]);
        } else {
            unsigned short h[8];
            for (int q = 0; q < 8; ++q) {
                const float x = q < per16 ? v[q] : 0.f;
                if (a.ab_format == 1) {
                    __nv_bfloat16 b = __float2bfloat16_rn(x);
                    h[q] = *reinterpret_cast<unsigned short*>(&b);
                } else {
                    __half b = __float2half_rn(x);
                    h[q] = *reinterpret_cast<unsigned short*>(&b);
                }
            }
            w = make_uint4(h[0] | (h[1] << 16), h[2] | (h[3] << 16), h[4] | (h[5] << 16), h[6] | (h[7] << 16));
        }
        *reinterpret_cast<uint4*>(dst) = w;
    }
}

// Band average of the per-bin COH, IMAGCOHY, PLV values.
__global__ void k_herk_band(HerkArgs a) {
    const FcCtrl* c = a.ctrl;
    if (c->bad) return;
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.P) return;
    const float invB = 1.0f / (float)(a.fsel1 - a.fsel0);
    for (int m = 0; m < 3; ++m) {
        const int mi = m == 0 ? MI_COH : m == 1 ? MI_IMAGCOHY : MI_PLV;
        if (!(a.mask & (1u << mi))) continue;
        float s = 0.f;
        for (int f = a.fsel0; f < a.fsel1; ++f) s = __fadd_rn(s, a.bins_out[((size_t)f * 3 + m) * a.P + p]);
        a.net[(size_t)mi * a.P + p] = __fmul_rn(s, invB);
    }
}

}  // namespace

cudaError_t launch_pack_operands(const PackArgs& a, cudaStream_t st) {
    k_pack_operands<<<152 * 8, 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_herk_tc(const HerkArgs& a, cudaStream_t st) {
    const int units = a.ntp * a.B;
    const int ctas = units < a.grid_ctas ? units : a.grid_ctas;
    cudaError_t e;
    if (a.ab_format == 2) {
        e = cudaFuncSetAttribute(k_herk_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
        if (e != cudaSuccess) return e;
        k_herk_tc<1><<<ctas, 128, SMEM_BYTES, st>>>(a);
    } else {
        e = cudaFuncSetAttribute(k_herk_tc<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
        if (e != cudaSuccess) return e;
        k_herk_tc<0><<<ctas, 128, SMEM_BYTES, st>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_herk_band(const HerkArgs& a, cudaStream_t st) {
    k_herk_band<<<(unsigned)((a.P + 255) / 256), 256, 0, st>>>(a);
    return cudaGetLastError();
}

size_t herk_chunk_bytes() { return CHUNK_BYTES; }
