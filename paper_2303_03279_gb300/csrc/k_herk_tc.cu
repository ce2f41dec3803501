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
// accumulation. COH, IMAGCOHY and PLV of the bin are finalized from TMEM and added to the
// band sums of the unit's bin group (the first bin stores, the later ones add with
// fire-and-forget reductions, red.global.add): one CTA walks all bins of a (tile pair, bin
// group) unit in order and each sum has one owner thread, so the additions land in bin order
// and the sums are reproducible. A small kernel adds the
// groups and scales by the number of bins. The non-linear sums
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
#include "tc.cuh"

#include <type_traits>

namespace {

using namespace fcmbar;
using namespace fctc;

constexpr int TILE = 128;             // nodes per tile (M = N = 128)
constexpr int CHUNK_BYTES = 16384;     // 128 rows x 128 bytes of K
constexpr int PHASE_OPS = 3;           // operand blocks per chunk of one phase (see k_herk_tc)
constexpr int STAGE_BYTES = PHASE_OPS * CHUNK_BYTES;
constexpr int NSTAGE = 4;              // chunk stages in flight
constexpr int EPI_WARPS = 8;           // epilogue warps: lane quarter w % 4, row nodes 64 (w / 4) ..
constexpr int SMEM_BYTES = NSTAGE * STAGE_BYTES + 512 + EPI_WARPS * 512;  // + barriers, TMEM address, 1/sqrt(PSD) rows per epilogue warp
constexpr uint32_t TMEM_COLS = 512;    // 2 phase buffers x 2 accumulators x 128 FP32 columns
constexpr int THREADS = 32 * EPI_WARPS + 32;  // warps 0-7: epilogue; warp 8: loads + MMAs

__device__ __forceinline__ long long packed_index(int i, int j, int n) {
    return (long long)i * n - (long long)i * (i + 1) / 2 + (j - i - 1);
}

__device__ __forceinline__ const unsigned char* op_block(const HerkArgs& a, int tile, int f, int kind, int chunk) {
    return a.ops + ((((size_t)tile * a.B + f) * 4 + kind) * a.nchunks + chunk) * (size_t)CHUNK_BYTES;
}

// Work of one CTA: units u = blockIdx.x + k gridDim.x of ntp x groups (tile pair u / groups,
// bin group u % groups), each over its bins in order, each bin in two phases.
struct HerkSeq {
    int u, f, fend;
};
__device__ __forceinline__ void seq_unit(const HerkArgs& a, HerkSeq& s, int u) {
    s.u = u;
    const int g = u % a.groups;
    s.f = a.fsel0 + g * a.group_bins;
    s.fend = min(a.fsel1, s.f + a.group_bins);
}
__device__ __forceinline__ void seq_next_bin(const HerkArgs& a, HerkSeq& s) {
    if (++s.f >= s.fend) seq_unit(a, s, s.u + (int)gridDim.x);
}

// Per (128-node tile pair, bin) step, two phases, each a pair of transposed products
// D^T[j][i] (TMEM lane = column node j of tile b, TMEM column = row node i of tile a):
//   phase A (CSD):     Re = XR_b XR_a^T,  Im = XR_b XI_a^T   -> COH, IMAGCOHY
//   phase B (phasors): Re = UR_b UR_a^T,  Im = UR_b UI_a^T   -> PLV
// Phase p accumulates in TMEM columns [256 p, 256 p + 256), so the epilogue of one phase
// runs while the tensor cores work on the next (warp-specialized: warp 8 lane 0 streams
// the operand chunks of the CTA's phase sequence through NSTAGE shared-memory stages and
// issues the MMAs; warps 0-7 drain TMEM, two per lane quarter, each over half of the row
// nodes). Every wait is bounded; a timeout is recorded in
// the control block.
template <int KIND>
__global__ void __launch_bounds__(THREADS, 1) k_herk_tc(HerkArgs a) {
    extern __shared__ __align__(1024) unsigned char smem[];
    FcCtrl* c = const_cast<FcCtrl*>(a.ctrl);
    if (c->bad) return;
    const int units = a.ntp * a.groups;
    if ((int)blockIdx.x >= units) return;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + NSTAGE * STAGE_BYTES);  // [NSTAGE]
    uint64_t* freeb = full + NSTAGE;                                             // [NSTAGE]
    uint64_t* accf = freeb + NSTAGE;                                             // [2] MMAs -> epilogue
    uint64_t* acce = accf + 2;                                                   // [2] epilogue -> MMAs
    uint64_t* drain = acce + 2;                                                  // [1]
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
    float* sinv_all = reinterpret_cast<float*>(smem + NSTAGE * STAGE_BYTES + 512);  // [EPI_WARPS][128]
    const int tid = threadIdx.x, warp = tid >> 5;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int s = 0; s < NSTAGE; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&freeb[s], 1);
        }
        mbar_init(&accf[0], 1);
        mbar_init(&accf[1], 1);
        mbar_init(&acce[0], EPI_WARPS);  // one arrival per epilogue warp
        mbar_init(&acce[1], EPI_WARPS);
        mbar_init(drain, 1);
        fence_mbar_init();
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;
    const long long wend = c->pushed + a.count;
    const int K = (int)(wend - ((a.W > 0 && wend > a.W) ? wend - a.W : 0));
    const float inv_K = 1.0f / (float)K;
    // this CTA's phase sequence: 2 per bin of each of its units
    int nphase = 0;
    for (int u = (int)blockIdx.x; u < units; u += (int)gridDim.x) {
        HerkSeq t;
        seq_unit(a, t, u);
        nphase += 2 * (t.fend - t.f);
    }
    bool failed = false;

    if (warp == EPI_WARPS) {
        // ---------------------------------------------------------- loads + MMAs
        if ((tid & 31) == 0) {
            const uint32_t idesc = make_idesc(KIND == 1 ? 2u : (a.ab_format == 1 ? 1u : 0u), TILE, TILE);
            const long long nchunk_total = (long long)nphase * a.nchunks;
            uint32_t full_ph[NSTAGE], free_ph[NSTAGE];
            for (int s = 0; s < NSTAGE; ++s) full_ph[s] = free_ph[s] = 0;
            uint32_t acce_ph[2] = {0, 0};
            long long loads = 0;
            HerkSeq ls;  // unit and bin of the phase being loaded
            seq_unit(a, ls, (int)blockIdx.x);
            long long lph = 0;
            auto issue_load = [&]() {  // chunk `loads` of the sequence into stage loads % NSTAGE
                if (loads >= nchunk_total) return;
                const int st = (int)(loads % NSTAGE);
                if (loads >= NSTAGE) {  // the MMAs of the chunk that used this stage have read it
                    if (!mbar_wait_bounded(&freeb[st], free_ph[st])) failed = true;
                    free_ph[st] ^= 1;
                }
                const long long ph = loads / a.nchunks;
                const int ch = (int)(loads % a.nchunks);
                for (; lph < ph; ++lph)
                    if (lph & 1) seq_next_bin(a, ls);  // after phase B: the next bin
                const int tp = ls.u / a.groups, f = ls.f;
                const int ta = a.tile_a[tp], tb = a.tile_b[tp];
                const int k0 = (ph & 1) ? 2 : 0;  // phase A: X operands, phase B: U operands
                unsigned char* dst = smem + st * STAGE_BYTES;
                mbar_expect_tx(&full[st], STAGE_BYTES);
                bulk_g2s(dst + 0 * CHUNK_BYTES, op_block(a, tb, f, k0, ch), CHUNK_BYTES, &full[st]);
                bulk_g2s(dst + 1 * CHUNK_BYTES, op_block(a, ta, f, k0, ch), CHUNK_BYTES, &full[st]);
                bulk_g2s(dst + 2 * CHUNK_BYTES, op_block(a, ta, f, k0 + 1, ch), CHUNK_BYTES, &full[st]);
                ++loads;
            };
            for (int s = 0; s < NSTAGE - 1; ++s) issue_load();
            long long consumed = 0;
            for (int ph = 0; ph < nphase && !failed; ++ph) {
                const int b = ph & 1;
                if (ph >= 2) {  // the epilogue has drained this TMEM half
                    if (!mbar_wait_bounded(&acce[b], acce_ph[b])) {
                        failed = true;
                        break;
                    }
                    acce_ph[b] ^= 1;
                    fence_after();
                }
                const uint32_t d = tmem + (uint32_t)(b * 2 * TILE);
                for (int ch = 0; ch < a.nchunks; ++ch) {
                    const int st = (int)(consumed % NSTAGE);
                    if (!mbar_wait_bounded(&full[st], full_ph[st])) {
                        failed = true;
                        break;
                    }
                    full_ph[st] ^= 1;
                    fence_after();
                    const uint32_t base = smem_u32(smem + st * STAGE_BYTES);
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks) {
                        const uint32_t acc = (ch > 0 || ks > 0) ? 1u : 0u;
                        const uint32_t off = ks * 256;
                        const uint64_t d_b = smem_desc(base + 0 * CHUNK_BYTES + off);   // XR_b or UR_b
                        const uint64_t d_ar = smem_desc(base + 1 * CHUNK_BYTES + off);  // XR_a or UR_a
                        const uint64_t d_ai = smem_desc(base + 2 * CHUNK_BYTES + off);  // XI_a or UI_a
                        mma<KIND>(d, d_b, d_ar, idesc, acc);
                        mma<KIND>(d + TILE, d_b, d_ai, idesc, acc);
                    }
                    mma_commit(&freeb[st]);  // the stage may be refilled once these MMAs have read it
                    ++consumed;
                    issue_load();            // refills the stage of the previous chunk
                }
                if (failed) break;
                mma_commit(&accf[b]);
            }
            // let every MMA and copy issued land before the CTA ends
            mma_commit(drain);
            mbar_wait_bounded(drain, 0);
            for (long long l = consumed; l < loads; ++l) {
                const int st = (int)(l % NSTAGE);
                mbar_wait_bounded(&full[st], full_ph[st]);
                full_ph[st] ^= 1;
            }
        }
    } else {
        // ---------------------------------------------------------- epilogue (warps 0-7)
        uint32_t accf_ph[2] = {0, 0};
        const int quarter = warp & 3, rhalf = warp >> 2;  // TMEM lanes 32 quarter ..; rows 64 rhalf ..
        const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
        float* sinv = sinv_all + warp * TILE;  // this warp's copy: no barrier across warps
        HerkSeq es;
        seq_unit(a, es, (int)blockIdx.x);
        for (int ph = 0; ph < nphase; ++ph) {
            const int b = ph & 1;
            if (ph > 0 && b == 0) seq_next_bin(a, es);
            const int tp = es.u / a.groups, f = es.f;
            const int ta = a.tile_a[tp], tb = a.tile_b[tp];
            const int j = tb * TILE + quarter * 32 + (tid & 31);  // this thread's TMEM lane: column node j
            if (b == 0) {  // 1/sqrt(PSD) of tile a's nodes, staged by this warp for itself
                __syncwarp();
                for (int r = 2 * rhalf; r < 2 * rhalf + 2; ++r) {  // the rows this warp reads
                    const int i = ta * TILE + r * 32 + (tid & 31);
                    sinv[r * 32 + (tid & 31)] = i < a.n ? a.inv_psd[(size_t)f * a.n + i] : 0.f;
                }
                __syncwarp();
            }
            // 1/sqrt(PSD) of this thread's column node, fetched while the MMAs run
            const float inv_j = (b == 0 && j < a.n) ? a.inv_psd[(size_t)f * a.n + j] : 0.f;
            // warp-uniform outcome: the TMEM loads below are warp-collective
            const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(&accf[b], accf_ph[b]) ? 1 : 0) != 0;
            accf_ph[b] ^= 1;
            if (!ok) {
                failed = true;
                break;
            }
            fence_after();
            const uint32_t col = (uint32_t)(b * 2 * TILE);
            float* out = a.part + (size_t)(es.u % a.groups) * 3 * a.P;  // this group's band sums
            // the unit's first bin writes its values, the later bins add to them (same thread,
            // same address: the reductions land after the store and in bin order)
            const bool first = f == a.fsel0 + (es.u % a.groups) * a.group_bins;
            // this warp's 64 row nodes: all eight loads (re and im of 4 x 16 columns) in flight
            // at once, one wait
            const int ibase = rhalf * (TILE / 2);
            uint32_t rre[4][16], rim[4][16];
#pragma unroll
            for (int s4 = 0; s4 < 4; ++s4) {
                tmem_ld16_issue(lane_base + col + ibase + 16 * s4, rre[s4]);
                tmem_ld16_issue(lane_base + col + TILE + ibase + 16 * s4, rim[s4]);
            }
            tmem_wait_ld();
#pragma unroll
            for (int s4 = 0; s4 < 4; ++s4) {
                tmem_keep(rre[s4]);
                tmem_keep(rim[s4]);
            }
            if (j < a.n) {
                // packed index of (i, j) for i = ta TILE + ibase, then p(i + 1) = p(i) + n - i - 2;
                // the unit's first bin stores, the later ones add (atomicAdd without its result:
                // a fire-and-forget reduction; same thread, same address, so in bin order)
                auto emit = [&](auto first_c) {
                    constexpr bool FIRST = decltype(first_c)::value;
                    int i = ta * TILE + ibase;
                    long long p = packed_index(i, j, a.n);
#pragma unroll
                    for (int s4 = 0; s4 < 4; ++s4) {
#pragma unroll
                        for (int q = 0; q < 16; ++q, p += a.n - i - 2, ++i) {
                            if (j <= i || i >= a.n) continue;
                            const float vre = __uint_as_float(rre[s4][q]), vim = __uint_as_float(rim[s4][q]);
                            float v0, v1 = 0.f;
                            long long o0;
                            if (b == 0) {
                                const float inv_i = sinv[ibase + 16 * s4 + q];
                                const float r = __fmul_rn(__fmul_rn(vre, inv_i), inv_j);
                                const float m = __fmul_rn(__fmul_rn(vim, inv_i), inv_j);
                                v0 = sqrtf(__fmaf_rn(r, r, __fmul_rn(m, m)));
                                v1 = m;
                                o0 = p;
                            } else {
                                v0 = __fmul_rn(sqrtf(__fmaf_rn(vre, vre, __fmul_rn(vim, vim))), inv_K);
                                o0 = 2 * a.P + p;
                            }
                            if (FIRST) {
                                out[o0] = v0;
                                if (b == 0) out[a.P + p] = v1;
                            } else {
                                atomicAdd(out + o0, v0);
                                if (b == 0) atomicAdd(out + a.P + p, v1);
                            }
                        }
                    }
                };
                if (first)
                    emit(std::true_type{});
                else
                    emit(std::false_type{});
            }
            fence_before();
            __syncwarp();
            if ((tid & 31) == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acce[b])) : "memory");
        }
    }
    fence_before();
    const int fail_any = __syncthreads_or(failed ? 1 : 0);
    fence_after();
    if (fail_any && tid == 0) atomicOr(&c->timeout, 1);
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

// ------------------------------------------------------------------ operand packing
// One thread per 16-byte row chunk of a core matrix position (tile, bin, node row m, 16-byte
// K unit), writing that chunk of all four operand kinds from one read of the spectra.
// Elements k of the 2K inner dimension: k < K -> trial k, first half; K <= k < 2K -> trial
// k - K, second half; beyond 2K -> 0.
//   XR = [Re X | Im X], XI = [Im X | -Re X], UR = [Re u | Im u], UI = [Im u | -Re u]
__device__ __forceinline__ float2 phasor_of_x(float2 X) {
    float m2 = __fmaf_rn(X.x, X.x, __fmul_rn(X.y, X.y));
    float r = (m2 > 0.0f) ? rsqrtf(m2) : 0.0f;
    return make_float2(__fmul_rn(X.x, r), __fmul_rn(X.y, r));
}

__device__ __forceinline__ uint4 pack_chunk(const float (&v)[8], int per16, int ab_format) {
    if (ab_format == 2) {  // TF32: round to nearest (ties away), stored in 32-bit words
        uint32_t t[4];
        for (int q = 0; q < 4; ++q) asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(t[q]) : "f"(v[q]));
        return make_uint4(t[0], t[1], t[2], t[3]);
    }
    unsigned short h[8];
    for (int q = 0; q < 8; ++q) {
        const float x = q < per16 ? v[q] : 0.f;
        if (ab_format == 1) {
            __nv_bfloat16 b = __float2bfloat16_rn(x);
            h[q] = *reinterpret_cast<unsigned short*>(&b);
        } else {
            __half b = __float2half_rn(x);
            h[q] = *reinterpret_cast<unsigned short*>(&b);
        }
    }
    return make_uint4(h[0] | (h[1] << 16), h[2] | (h[3] << 16), h[4] | (h[5] << 16), h[6] | (h[7] << 16));
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
    const long long total = (long long)a.ntiles * a.B * a.nchunks * units_per_block;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        long long rest = e;
        const int r = (int)(rest % 8); rest /= 8;       // row within core matrix
        const int kc = (int)(rest % 8); rest /= 8;      // core matrix along K within the chunk
        const int m8 = (int)(rest % 16); rest /= 16;    // 8-row group
        const int ch = (int)(rest % a.nchunks); rest /= a.nchunks;
        const int f = (int)(rest % a.B); rest /= a.B;
        const int tile = (int)rest;
        const int m = m8 * 8 + r;
        const int node = tile * TILE + m;
        const int k0 = (ch * 8 + kc) * per16;           // first inner index of this 16-byte unit
        float v[4][8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int k = k0 + q;
            v[0][q] = v[1][q] = v[2][q] = v[3][q] = 0.f;  // padding: +0 exactly
            if (q < per16 && node < a.n && k < 2 * K) {
                const int part = k >= K;
                const long long trial = start + (part ? k - K : k);
                const float2 X = a.ring[((size_t)(trial % a.slots) * a.B + f) * a.n + node];
                const float2 u = phasor_of_x(X);
                v[0][q] = part ? X.y : X.x;   // XR
                v[1][q] = part ? -X.x : X.y;  // XI
                v[2][q] = part ? u.y : u.x;   // UR
                v[3][q] = part ? -u.x : u.y;  // UI
            }
        }
#pragma unroll
        for (int kind = 0; kind < 4; ++kind) {
            unsigned char* dst = a.ops + ((((size_t)tile * a.B + f) * 4 + kind) * a.nchunks + ch) * (size_t)CHUNK_BYTES +
                                 (size_t)(m8 * 8 + kc) * 128 + r * 16;
            *reinterpret_cast<uint4*>(dst) = pack_chunk(v[kind], per16, a.ab_format);
        }
    }
}

// Band average of COH, IMAGCOHY, PLV: the bin groups' sums added in group order, times 1/bins.
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
        for (int g = 0; g < a.groups; ++g) s = __fadd_rn(s, a.part[((size_t)g * 3 + m) * a.P + p]);
        a.net[(size_t)mi * a.P + p] = __fmul_rn(s, invB);
    }
}

}  // namespace

cudaError_t launch_pack_operands(const PackArgs& a, cudaStream_t st) {
    k_pack_operands<<<fc_device_sms() * 8, 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_herk_tc(const HerkArgs& a, cudaStream_t st) {
    const int units = a.ntp * a.groups;
    const int ctas = units < a.grid_ctas ? units : a.grid_ctas;
    cudaError_t e;
    if (a.ab_format == 2) {
        e = cudaFuncSetAttribute(k_herk_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
        if (e != cudaSuccess) return e;
        k_herk_tc<1><<<ctas, THREADS, SMEM_BYTES, st>>>(a);
    } else {
        e = cudaFuncSetAttribute(k_herk_tc<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
        if (e != cudaSuccess) return e;
        k_herk_tc<0><<<ctas, THREADS, SMEM_BYTES, st>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_herk_band(const HerkArgs& a, cudaStream_t st) {
    k_herk_band<<<(unsigned)((a.P + 255) / 256), 256, 0, st>>>(a);
    return cudaGetLastError();
}

size_t herk_chunk_bytes() { return CHUNK_BYTES; }
