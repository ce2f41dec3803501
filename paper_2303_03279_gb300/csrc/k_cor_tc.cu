// k_cor_tc.cu - COR (Supplementary Information 1, Time Domain: Pearson correlation of the
// trial's node signals, averaged over the window's trials) on the 5th-generation tensor
// cores.
//
// With z_i the normalized trial of node i (k_cor_normalize), COR_k(i, j) = z_i . z_j: per
// trial a symmetric rank-N product Z Z^T over the upper triangle of 128-node tiles. FP32
// accuracy from TF32 operands by splitting z = hi + lo (hi = z rounded to TF32, lo = the
// rest rounded to TF32) and summing hi_j hi_i + hi_j lo_i + lo_j hi_i (the dropped lo lo
// term is below 2^-22 of the product). Per 128-node tile pair, each trial's 128 x 128 block
// accumulates over its N samples in FP32 in TMEM (tcgen05.mma kind::tf32, M = N = 128,
// products transposed: TMEM lane = column node j, TMEM column = row node i); eight epilogue
// warps then add the block into per-pair double-float running sums held in registers
// (lazy TwoSum), so sums over many trials keep FP64-class accuracy. A trial's values are
// the same whether it is added (when pushed) or subtracted (when it leaves the window):
// the same operand blocks go through the same MMA sequence.
//
// Operand ring (built once per trial by k_cor_tc_pack): for each trial slot, 128-node tile
// and 32-sample chunk, the hi and the lo block (16 KB each, K-major canonical core-matrix
// layout: 8 rows x 16 bytes, leading stride 128 B, 8-row-group stride 1024 B), adjacent, so
// one 32 KB bulk copy fetches both.
#include "df32.cuh"
#include "fc_internal.h"
#include "mbar.cuh"
#include "tc.cuh"

namespace {

using namespace fcmbar;
using namespace fctc;

constexpr int TILE = 128;
constexpr int CHUNK_SAMPLES = 32;              // TF32 samples per 128-byte K-chunk
constexpr int BLOCK_BYTES = 16384;             // 128 rows x 128 bytes
constexpr int PAIR_BYTES = 2 * BLOCK_BYTES;    // hi and lo of one tile and chunk
constexpr int STAGE_BYTES = 2 * PAIR_BYTES;    // both tiles
constexpr int NSTAGE = 3;
constexpr int EPI_WARPS = 8;                   // lane quarter w % 4, row nodes 64 (w / 4) ..
constexpr int THREADS = 32 * EPI_WARPS + 32;   // warp 8: loads + MMAs
constexpr uint32_t TMEM_COLS = 256;            // two trial buffers x 128 FP32 columns
constexpr int SMEM_BYTES = NSTAGE * STAGE_BYTES + 256;

__device__ __forceinline__ long long packed_index(int i, int j, int n) {
    return (long long)i * n - (long long)i * (i + 1) / 2 + (j - i - 1);
}

__device__ __forceinline__ void tile_pair(int tp, int nt, int& ta, int& tb) {
    int r = tp, a = 0;
    while (r >= nt - a) {
        r -= nt - a;
        ++a;
    }
    ta = a;
    tb = a + r;
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t t;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(t) : "f"(x));
    return t;
}

// One thread per 16-byte unit (4 samples of one node row) of the trials written by this call.
__global__ void k_cor_tc_pack(CorTcArgs a) {
    const FcCtrl* c = a.ctrl;
    if (c->bad) return;
    const int ntr = a.count - a.write_from;
    const long long total = (long long)ntr * a.nt * a.nchunks * TILE * 8;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        long long rest = e;
        const int r = (int)(rest % 8); rest /= 8;     // row within the core matrix
        const int kc = (int)(rest % 8); rest /= 8;    // 16-byte unit along K
        const int m8 = (int)(rest % 16); rest /= 16;  // 8-row group
        const int ch = (int)(rest % a.nchunks); rest /= a.nchunks;
        const int tile = (int)(rest % a.nt); rest /= a.nt;
        const int tr = a.write_from + (int)rest;
        const int slot = (int)((c->pushed + tr) % a.slots);
        const int node = tile * TILE + m8 * 8 + r;
        const int t0 = ch * CHUNK_SAMPLES + kc * 4;
        uint32_t hi[4], lo[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int t = t0 + q;
            const float z = (node < a.n && t < a.N) ? a.zring[((size_t)slot * a.n + node) * a.N + t] : 0.f;
            hi[q] = to_tf32(z);
            lo[q] = to_tf32(__fsub_rn(z, __uint_as_float(hi[q])));  // exact difference, then rounded
        }
        unsigned char* dst = a.ops + (((size_t)slot * a.nt + tile) * a.nchunks + ch) * (size_t)PAIR_BYTES +
                             (size_t)(m8 * 8 + kc) * 128 + r * 16;
        *reinterpret_cast<uint4*>(dst) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
        *reinterpret_cast<uint4*>(dst + BLOCK_BYTES) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
    }
}

// Trials of one unit. Mode 0 (stream push): the newest trial (+1) and, once the window is
// full, the trial leaving it (-1). Mode 1 (window): group g's share of the window's trials.
struct UnitTrials {
    long long first;  // trial index of entry 0 (mode 1) or the newest trial (mode 0)
    int count;
};
__device__ __forceinline__ UnitTrials unit_trials(const CorTcArgs& a, int u, long long start, long long end) {
    UnitTrials t;
    if (a.mode == 0) {
        t.first = end - 1;
        t.count = (a.W > 0 && end - 1 >= a.W) ? 2 : 1;
    } else {
        const long long K = end - start;
        const long long tg = (K + a.groups - 1) / a.groups;
        const int g = u / a.ntp;
        const long long k0 = start + g * tg;
        const long long k1 = k0 + tg < end ? k0 + tg : end;
        t.first = k0;
        t.count = k1 > k0 ? (int)(k1 - k0) : 0;
    }
    return t;
}
__device__ __forceinline__ long long entry_trial(const CorTcArgs& a, const UnitTrials& t, int q) {
    return a.mode == 0 ? (q == 0 ? t.first : t.first - a.W) : t.first + q;
}

__global__ void __launch_bounds__(THREADS, 1) k_cor_tc(CorTcArgs a) {
    extern __shared__ __align__(1024) unsigned char smem[];
    FcCtrl* c = const_cast<FcCtrl*>(a.ctrl);
    if (c->bad) return;
    const int units = a.mode == 0 ? a.ntp : a.ntp * a.groups;
    if ((int)blockIdx.x >= units) return;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + NSTAGE * STAGE_BYTES);  // [NSTAGE]
    uint64_t* freeb = full + NSTAGE;                                             // [NSTAGE]
    uint64_t* accf = freeb + NSTAGE;                                             // [2] MMAs -> epilogue
    uint64_t* acce = accf + 2;                                                   // [2] epilogue -> MMAs
    uint64_t* drain = acce + 2;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
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
        mbar_init(&acce[0], EPI_WARPS);
        mbar_init(&acce[1], EPI_WARPS);
        mbar_init(drain, 1);
        fence_mbar_init();
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;
    const long long end = c->pushed + a.count;
    const long long start = (a.W > 0 && end > a.W) ? end - a.W : 0;
    const int my_units = (units - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
    bool failed = false;

    if (warp == EPI_WARPS) {
        // ---------------------------------------------------------- loads + MMAs
        if ((tid & 31) == 0) {
            const uint32_t idesc = make_idesc(2u, TILE, TILE);
            uint32_t full_ph[NSTAGE], free_ph[NSTAGE];
            for (int s = 0; s < NSTAGE; ++s) full_ph[s] = free_ph[s] = 0;
            uint32_t acce_ph[2] = {0, 0};
            // load cursor over (unit m, entry q, chunk ch) of this CTA, ahead of the MMAs
            int lm = 0, lq = 0, lch = 0;
            UnitTrials lt = unit_trials(a, (int)blockIdx.x, start, end);
            auto lskip = [&]() {  // move past units without trials
                while (lm < my_units && lq >= lt.count) {
                    ++lm;
                    lq = 0;
                    lch = 0;
                    if (lm < my_units) lt = unit_trials(a, (int)blockIdx.x + lm * (int)gridDim.x, start, end);
                }
            };
            lskip();
            long long loads = 0;
            auto issue_load = [&]() {
                if (lm >= my_units) return;
                const int st = (int)(loads % NSTAGE);
                if (loads >= NSTAGE) {  // the MMAs of the chunk that used this stage have read it
                    if (!mbar_wait_bounded(&freeb[st], free_ph[st])) failed = true;
                    free_ph[st] ^= 1;
                }
                const int u = (int)blockIdx.x + lm * (int)gridDim.x;
                int ta, tb;
                tile_pair(u % a.ntp, a.nt, ta, tb);
                const int slot = (int)(entry_trial(a, lt, lq) % a.slots);
                const unsigned char* src = a.ops + ((size_t)slot * a.nt) * a.nchunks * (size_t)PAIR_BYTES;
                unsigned char* dst = smem + st * STAGE_BYTES;
                mbar_expect_tx(&full[st], STAGE_BYTES);
                bulk_g2s(dst, src + ((size_t)tb * a.nchunks + lch) * PAIR_BYTES, PAIR_BYTES, &full[st]);
                bulk_g2s(dst + PAIR_BYTES, src + ((size_t)ta * a.nchunks + lch) * PAIR_BYTES, PAIR_BYTES, &full[st]);
                ++loads;
                if (++lch == a.nchunks) {
                    lch = 0;
                    ++lq;
                    lskip();
                }
            };
            for (int s = 0; s < NSTAGE - 1; ++s) issue_load();
            long long consumed = 0;
            int ph = 0;  // trial entries processed by this CTA (TMEM buffer ph & 1)
            for (int m = 0; m < my_units && !failed; ++m) {
                const UnitTrials ut = unit_trials(a, (int)blockIdx.x + m * (int)gridDim.x, start, end);
                for (int q = 0; q < ut.count && !failed; ++q, ++ph) {
                    const int b = ph & 1;
                    if (ph >= 2) {  // the epilogue has drained this buffer
                        if (!mbar_wait_bounded(&acce[b], acce_ph[b])) {
                            failed = true;
                            break;
                        }
                        acce_ph[b] ^= 1;
                        fence_after();
                    }
                    const uint32_t d = tmem + (uint32_t)(b * TILE);
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
                            const uint32_t off = ks * 256;
                            const uint64_t bh = smem_desc(base + off);                              // z_hi, tile b
                            const uint64_t bl = smem_desc(base + BLOCK_BYTES + off);                // z_lo, tile b
                            const uint64_t ah = smem_desc(base + PAIR_BYTES + off);                 // z_hi, tile a
                            const uint64_t al = smem_desc(base + PAIR_BYTES + BLOCK_BYTES + off);   // z_lo, tile a
                            mma<1>(d, bh, ah, idesc, (ch > 0 || ks > 0) ? 1u : 0u);
                            mma<1>(d, bh, al, idesc, 1u);
                            mma<1>(d, bl, ah, idesc, 1u);
                        }
                        mma_commit(&freeb[st]);
                        ++consumed;
                        issue_load();
                    }
                    if (failed) break;
                    mma_commit(&accf[b]);
                }
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
        const int quarter = warp & 3, rhalf = warp >> 2;
        const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
        int ph = 0;
        for (int m = 0; m < my_units && !failed; ++m) {
            const int u = (int)blockIdx.x + m * (int)gridDim.x;
            int ta, tb;
            tile_pair(u % a.ntp, a.nt, ta, tb);
            const int j = tb * TILE + quarter * 32 + (tid & 31);
            const int i0 = ta * TILE + rhalf * (TILE / 2);
            const UnitTrials ut = unit_trials(a, u, start, end);
            float hi[64], lo[64];
#pragma unroll
            for (int r = 0; r < 64; ++r) {
                hi[r] = lo[r] = 0.f;
                const int i = i0 + r;
                if (a.mode == 0 && i < j && j < a.n) {
                    const long long id = packed_index(i, j, a.n);
                    hi[r] = a.cor_acc[id];
                    lo[r] = a.cor_acc[a.P + id];
                }
            }
            for (int q = 0; q < ut.count; ++q, ++ph) {
                const int b = ph & 1;
                // warp-uniform outcome: the TMEM loads below are warp-collective
                const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(&accf[b], accf_ph[b]) ? 1 : 0) != 0;
                accf_ph[b] ^= 1;
                if (!ok) {
                    failed = true;
                    break;
                }
                fence_after();
                const bool neg = a.mode == 0 && q == 1;  // the trial leaving the window
                const uint32_t col = (uint32_t)(b * TILE + rhalf * (TILE / 2));
#pragma unroll
                for (int c0 = 0; c0 < 64; c0 += 16) {
                    float v[16];
                    tmem_ld16(lane_base + col + c0, v);
#pragma unroll
                    for (int r = 0; r < 16; ++r) {
                        float s, e;
                        two_sum(hi[c0 + r], neg ? -v[r] : v[r], s, e);
                        hi[c0 + r] = s;
                        lo[c0 + r] = __fadd_rn(lo[c0 + r], e);
                    }
                }
                fence_before();
                __syncwarp();
                if ((tid & 31) == 0)
                    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acce[b])) : "memory");
            }
            if (failed) break;
            const long long K = end - start;
            const float invK = K > 0 ? 1.0f / (float)K : 0.f;
            const bool partial = a.mode == 1 && a.groups > 1;
            const int g = u / a.ntp;
#pragma unroll
            for (int r = 0; r < 64; ++r) {
                const int i = i0 + r;
                if (!(i < j && j < a.n)) continue;
                float s, e;
                two_sum(hi[r], lo[r], s, e);  // back to a normalized double word
                const long long id = packed_index(i, j, a.n);
                if (partial) {
                    a.part[(2 * (size_t)g) * a.P + id] = s;
                    a.part[(2 * (size_t)g + 1) * a.P + id] = e;
                    continue;
                }
                a.cor_acc[id] = s;
                a.cor_acc[a.P + id] = e;
                if (a.finalize) a.net[id] = __fmul_rn(__fadd_rn(s, e), invK);
            }
        }
    }
    fence_before();
    const int fail_any = __syncthreads_or(failed ? 1 : 0);
    fence_after();
    if (fail_any && tid == 0) atomicOr(&c->timeout, 1);
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

}  // namespace

cudaError_t launch_cor_tc_pack(const CorTcArgs& a, cudaStream_t st) {
    if (a.count - a.write_from <= 0) return cudaSuccess;
    k_cor_tc_pack<<<fc_device_sms() * 8, 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_cor_tc(const CorTcArgs& a, cudaStream_t st) {
    if (a.mode != 0 && a.mode != 1) return cudaErrorInvalidValue;
    if (a.groups < 1 || (a.groups > 1 && (a.mode != 1 || !a.part))) return cudaErrorInvalidValue;
    const int units = a.mode == 0 ? a.ntp : a.ntp * a.groups;
    if (units <= 0) return cudaSuccess;
    const int ctas = units < a.grid_ctas ? units : a.grid_ctas;
    cudaError_t e = cudaFuncSetAttribute(k_cor_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    if (e != cudaSuccess) return e;
    k_cor_tc<<<ctas, THREADS, SMEM_BYTES, st>>>(a);
    return cudaGetLastError();
}

size_t cor_tc_pair_bytes() { return PAIR_BYTES; }
