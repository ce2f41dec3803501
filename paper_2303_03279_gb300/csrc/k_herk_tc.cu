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
// accumulation; split TF32 (ab_format 3) stores each operand as a TF32 high part and a TF32
// low part (operand kinds 4 .. 7) and forms every product as hi hi + hi lo + lo hi, which
// keeps the sums FP32-class. COH, IMAGCOHY and PLV of the bin are finalized from TMEM and added to the
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
// One cp.async.bulk moves a block into shared memory as is. Short last chunk (operands of
// the resident-operand form, last_kc < 8): the last K-chunk keeps only its first last_kc
// core-matrix columns, those up to the last K-step that holds inner positions (the others
// hold zero padding only), as (m / 8) * last_kc + kc core matrices, 8-row groups last_kc x
// 128 B apart, at the start of its 16 KB block; its copies move 2 KB per column and its
// MMAs take last_kc / 2 K-steps.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "df32.cuh"
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

// Operand kinds per (tile, bin): XR, XI, UR, UI; split TF32 (ab_format 3) adds their
// low parts as kinds 4 .. 7.
__device__ __forceinline__ int op_kinds(int ab_format) { return ab_format == 3 ? 8 : 4; }

__device__ __forceinline__ const unsigned char* op_block(const HerkArgs& a, int tile, int f, int kind, int chunk) {
    return a.ops + ((((size_t)tile * a.B + f) * op_kinds(a.ab_format) + kind) * a.nchunks + chunk) * (size_t)CHUNK_BYTES;
}

// Core-matrix columns stored in K-chunk ch of a pack with last_kc (the short layout of the
// last chunk when 2 <= last_kc < 8, else all 8).
__device__ __forceinline__ int chunk_cols(int last_kc, int ch, int nchunks) {
    return (ch == nchunks - 1 && last_kc >= 2 && last_kc < 8) ? last_kc : 8;
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
// SPLIT (split TF32, KIND 1): each operand is a TF32 high part and a TF32 low part (the
// rounding residue); a stage holds both (six blocks), and each K step issues three MMAs,
// hi x hi + hi x lo + lo x hi, so the products keep FP32-class accuracy (the dropped lo x lo
// term and the low part's own rounding are ~2^-22 of the product).
template <bool SPLIT>
struct HerkStages {
    static constexpr int NST = SPLIT ? 2 : NSTAGE;                       // stages in flight
    static constexpr int SB = (SPLIT ? 2 : 1) * STAGE_BYTES;             // bytes per stage
    static constexpr int SMEM = NST * SB + 512 + EPI_WARPS * 512;
};

template <int KIND, bool SPLIT>
__global__ void __launch_bounds__(THREADS, 1) k_herk_tc(HerkArgs a) {
    constexpr int NST = HerkStages<SPLIT>::NST, SB = HerkStages<SPLIT>::SB;
    extern __shared__ __align__(1024) unsigned char smem[];
    FcCtrl* c = const_cast<FcCtrl*>(a.ctrl);
    if (c->bad) return;
    const int units = a.ntp * a.groups;
    if ((int)blockIdx.x >= units) return;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + NST * SB);  // [NST]
    uint64_t* freeb = full + NST;                                    // [NST]
    uint64_t* accf = freeb + NST;                                    // [2] MMAs -> epilogue
    uint64_t* acce = accf + 2;                                       // [2] epilogue -> MMAs
    uint64_t* drain = acce + 2;                                      // [1]
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
    float* sinv_all = reinterpret_cast<float*>(smem + NST * SB + 512);  // [EPI_WARPS][128]
    const int tid = threadIdx.x, warp = tid >> 5;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int s = 0; s < NST; ++s) {
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
            // N = 256: the row tile's two kinds (XR_a then XI_a, or UR_a then UI_a) are adjacent
            // in shared memory with the 8-row-group stride, so one MMA takes both as a
            // 256-row operand and writes both accumulators (TMEM columns 0-127 and 128-255)
            const uint32_t idesc = make_idesc(KIND == 1 ? 2u : (a.ab_format == 1 ? 1u : 0u), TILE, 2 * TILE);
            const long long nchunk_total = (long long)nphase * a.nchunks;
            uint32_t full_ph[NST], free_ph[NST];
            for (int s = 0; s < NST; ++s) full_ph[s] = free_ph[s] = 0;
            uint32_t acce_ph[2] = {0, 0};
            long long loads = 0;
            HerkSeq ls;  // unit and bin of the phase being loaded
            seq_unit(a, ls, (int)blockIdx.x);
            long long lph = 0;
            auto issue_load = [&]() {  // chunk `loads` of the sequence into stage loads % NST
                if (loads >= nchunk_total) return;
                const int st = (int)(loads % NST);
                if (loads >= NST) {  // the MMAs of the chunk that used this stage have read it
                    if (!mbar_wait_bounded(&freeb[st], free_ph[st])) failed = true;
                    free_ph[st] ^= 1;
                }
                const long long ph = loads / a.nchunks;
                const int ch = (int)(loads % a.nchunks);
                for (; lph < ph; ++lph)
                    if (lph & 1) seq_next_bin(a, ls);  // after phase B: the next bin
                const int tp = a.tp0 + ls.u / a.groups, f = ls.f;
                const int ta = a.tile_a[tp], tb = a.tile_b[tp];
                const int k0 = (ph & 1) ? 2 : 0;  // phase A: X operands, phase B: U operands
                unsigned char* dst = smem + st * SB;
                mbar_expect_tx(&full[st], SB);
                bulk_g2s(dst + 0 * CHUNK_BYTES, op_block(a, tb, f, k0, ch), CHUNK_BYTES, &full[st]);
                bulk_g2s(dst + 1 * CHUNK_BYTES, op_block(a, ta, f, k0, ch), CHUNK_BYTES, &full[st]);
                bulk_g2s(dst + 2 * CHUNK_BYTES, op_block(a, ta, f, k0 + 1, ch), CHUNK_BYTES, &full[st]);
                if constexpr (SPLIT) {  // the low parts, in the same order
                    bulk_g2s(dst + 3 * CHUNK_BYTES, op_block(a, tb, f, k0 + 4, ch), CHUNK_BYTES, &full[st]);
                    bulk_g2s(dst + 4 * CHUNK_BYTES, op_block(a, ta, f, k0 + 4, ch), CHUNK_BYTES, &full[st]);
                    bulk_g2s(dst + 5 * CHUNK_BYTES, op_block(a, ta, f, k0 + 5, ch), CHUNK_BYTES, &full[st]);
                }
                ++loads;
            };
            for (int s = 0; s < NST - 1; ++s) issue_load();
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
                    const int st = (int)(consumed % NST);
                    if (!mbar_wait_bounded(&full[st], full_ph[st])) {
                        failed = true;
                        break;
                    }
                    full_ph[st] ^= 1;
                    fence_after();
                    const uint32_t base = smem_u32(smem + st * SB);
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks) {
                        const uint32_t acc = (ch > 0 || ks > 0) ? 1u : 0u;
                        const uint32_t off = ks * 256;
                        const uint64_t d_b = smem_desc(base + 0 * CHUNK_BYTES + off);   // XR_b or UR_b
                        const uint64_t d_a2 = smem_desc(base + 1 * CHUNK_BYTES + off);  // [XR_a; XI_a] or [UR_a; UI_a]
                        mma<KIND>(d, d_b, d_a2, idesc, acc);
                        if constexpr (SPLIT) {
                            const uint64_t d_bl = smem_desc(base + 3 * CHUNK_BYTES + off);
                            const uint64_t d_a2l = smem_desc(base + 4 * CHUNK_BYTES + off);
                            mma<KIND>(d, d_b, d_a2l, idesc, 1u);   // hi x lo
                            mma<KIND>(d, d_bl, d_a2, idesc, 1u);   // lo x hi
                        }
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
                const int st = (int)(l % NST);
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
        // 1/sqrt(PSD) of the next bin's nodes (this warp's two row groups of tile a and this
        // thread's column node of tile b), loaded one bin ahead so that no phase waits on them
        float pf_i[2], pf_j;
        auto prefetch = [&](const HerkSeq& t) {
            pf_i[0] = pf_i[1] = pf_j = 0.f;
            if (t.u >= units) return;
            const int ptp = a.tp0 + t.u / a.groups;
            const int pta = a.tile_a[ptp], ptb = a.tile_b[ptp];
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const int i = pta * TILE + (2 * rhalf + r) * 32 + (tid & 31);
                if (i < a.n) pf_i[r] = a.inv_psd[(size_t)t.f * a.n + i];
            }
            const int jj = ptb * TILE + quarter * 32 + (tid & 31);
            if (jj < a.n) pf_j = a.inv_psd[(size_t)t.f * a.n + jj];
        };
        prefetch(es);
        float inv_j = 0.f;
        for (int ph = 0; ph < nphase; ++ph) {
            const int b = ph & 1;
            if (ph > 0 && b == 0) seq_next_bin(a, es);
            const int tp = a.tp0 + es.u / a.groups, f = es.f;
            const int ta = a.tile_a[tp], tb = a.tile_b[tp];
            const int j = tb * TILE + quarter * 32 + (tid & 31);  // this thread's TMEM lane: column node j
            if (b == 0) {  // this bin's 1/sqrt(PSD), staged by this warp for itself; next bin's fetched
                __syncwarp();
                sinv[(2 * rhalf) * 32 + (tid & 31)] = pf_i[0];
                sinv[(2 * rhalf + 1) * 32 + (tid & 31)] = pf_i[1];
                inv_j = pf_j;
                __syncwarp();
                HerkSeq nx = es;
                seq_next_bin(a, nx);
                prefetch(nx);
            }
            // warp-uniform outcome: the TMEM loads below are warp-collective
            const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(&accf[b], accf_ph[b]) ? 1 : 0) != 0;
            accf_ph[b] ^= 1;
            if (!ok) {
                failed = true;
                break;
            }
            fence_after();
            const uint32_t col = (uint32_t)(b * 2 * TILE);
            // this group's band sums (none in accumulator mode)
            float* out = a.acc_out ? nullptr : a.part + (size_t)(es.u % a.groups) * 3 * a.P;
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
            if (a.acc_out && j < a.n) {
                // accumulator mode: the raw sums of pair (i, j) (i < j) into the streaming
                // accumulator block of its 32-node tile pair, word (i % 32) 32 + j % 32: phase A the
                // CSD real part (field 0), phase B the phasor sums (fields 2, 3); hi word the
                // FP32 sum, lo word 0
                const int tb32 = j >> 5;
#pragma unroll
                for (int s4 = 0; s4 < 4; ++s4) {
                    const int i0 = ta * TILE + ibase + 16 * s4;
                    const int ta32 = i0 >> 5;
                    const long long tp32 = (long long)ta32 * a.nt32 - (long long)ta32 * (ta32 - 1) / 2 + (tb32 - ta32);
                    float* blk = a.acc_out + ((size_t)tp32 * a.B + f) * FC_BLOCK_WORDS;
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const int i = i0 + q;
                        if (j <= i || i >= a.n) continue;
                        const int w = (i & 31) * 32 + (j & 31);
                        const float vre = __uint_as_float(rre[s4][q]), vim = __uint_as_float(rim[s4][q]);
                        if (b == 0) {
                            blk[0 * FC_TT + w] = vre;
                            blk[1 * FC_TT + w] = 0.f;
                        } else {
                            blk[4 * FC_TT + w] = vre;
                            blk[5 * FC_TT + w] = 0.f;
                            blk[6 * FC_TT + w] = vim;
                            blk[7 * FC_TT + w] = 0.f;
                        }
                    }
                }
            } else if (j < a.n) {
                // packed index of (i, j) for i = ta TILE + ibase, then p(i + 1) = p(i) + n - i - 2
                // (below 2^31: n < 65536); the unit's first bin stores, the later ones add
                // (atomicAdd without its result: a fire-and-forget reduction; same thread, same
                // address, so in bin order). Off-diagonal tile pairs (ta < tb) have i < j < n for
                // every element (tile a is not the last tile): no per-element test there.
                // |z| = t rsqrt(t) with t = |z|^2 (a few ulp, far inside the tensor-core error).
                auto emit = [&](auto first_c, auto full_c) {
                    constexpr bool FIRST = decltype(first_c)::value;
                    constexpr bool FULL = decltype(full_c)::value;
                    int i = ta * TILE + ibase;
                    int p = (int)packed_index(i, j, a.n);
                    float* o_a = out + (b == 0 ? 0 : 2 * a.P);
#pragma unroll
                    for (int s4 = 0; s4 < 4; ++s4) {
#pragma unroll
                        for (int q = 0; q < 16; ++q, p += a.n - i - 2, ++i) {
                            if (!FULL && (j <= i || i >= a.n)) continue;
                            const float vre = __uint_as_float(rre[s4][q]), vim = __uint_as_float(rim[s4][q]);
                            if (b == 0) {
                                const float sc = __fmul_rn(sinv[ibase + 16 * s4 + q], inv_j);
                                const float r = __fmul_rn(vre, sc), m = __fmul_rn(vim, sc);
                                const float t = __fmaf_rn(r, r, __fmul_rn(m, m));
                                const float coh = t > 0.f ? __fmul_rn(t, rsqrtf(t)) : 0.f;
                                if (FIRST) {
                                    o_a[p] = coh;
                                    o_a[a.P + p] = m;
                                } else {
                                    atomicAdd(o_a + p, coh);
                                    atomicAdd(o_a + a.P + p, m);
                                }
                            } else {
                                const float t = __fmaf_rn(vre, vre, __fmul_rn(vim, vim));
                                const float plv = t > 0.f ? __fmul_rn(__fmul_rn(t, rsqrtf(t)), inv_K) : 0.f;
                                if (FIRST)
                                    o_a[p] = plv;
                                else
                                    atomicAdd(o_a + p, plv);
                            }
                        }
                    }
                };
                const bool full = ta < tb;
                if (first) {
                    if (full)
                        emit(std::true_type{}, std::true_type{});
                    else
                        emit(std::true_type{}, std::false_type{});
                } else {
                    if (full)
                        emit(std::false_type{}, std::true_type{});
                    else
                        emit(std::false_type{}, std::false_type{});
                }
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

// ------------------------------------------------------- resident-operand form
// The same products with one row tile's operands held in shared memory: a work item is
// (row tile a, column tiles b0 .. b1 - 1, bin group, phase). For each bin of the group the
// two row-side operand kinds of tile a (XR_a, XI_a in phase A; UR_a, UI_a in phase B) are
// loaded once into resident slots, and the column-side operand of each tile b (XR_b or
// UR_b) streams through NST 16 KB stages: per (tile pair, bin, phase) 64 KB of operands
// move instead of 192 KB. Warp 8 issues the bulk copies, warp 9 the MMAs, warps 0-7 drain
// TMEM (two buffers, so one unit's epilogue overlaps the next unit's MMAs). A unit's band
// sums are written by one CTA in bin order, as in k_herk_tc.
constexpr int RC_MAX = 4;                                   // resident K-chunks (2K <= 256 BF16 values)
constexpr int NST = 5;                                      // streaming stages of one 16 KB block
constexpr int RES_BYTES = RC_MAX * 2 * CHUNK_BYTES;         // 128 KB
constexpr int RES_EPI = 8;                                  // epilogue warps: lane quarter w % 4, 64 rows each
constexpr int RES_ROWS = TILE * 4 / RES_EPI;                // row nodes per epilogue warp
constexpr int RES_SMEM = RES_BYTES + NST * CHUNK_BYTES + 1024 + RES_EPI * 4 * RES_ROWS;
constexpr int RES_THREADS = 32 * RES_EPI + 64;              // warps 0-15 epilogue, 16 copies, 17 MMAs

// sqrt(x), x >= 0, with the hardware approximation (relative error near 2^-23; 0 for 0).
__device__ __forceinline__ float sqrt_approx(float x) {
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

struct ResItem {
    int a, b0, b1, p, g, f0, f1;
};
__device__ __forceinline__ ResItem res_item(const HerkArgs& A, int it) {
    ResItem r;
    const int per_p = A.groups * A.nseg;
    r.p = it / per_p;
    const int rem = it - r.p * per_p;
    r.g = rem / A.nseg;
    const int sg = rem - r.g * A.nseg;
    r.a = A.seg_a[sg];
    r.b0 = A.seg_b0[sg];
    r.b1 = A.seg_b1[sg];
    r.f0 = A.fsel0 + r.g * A.group_bins;
    r.f1 = min(A.fsel1, r.f0 + A.group_bins);
    return r;
}

template <int KIND>
__global__ void __launch_bounds__(RES_THREADS, 1) k_herk_res(HerkArgs a) {
    constexpr int EPI = RES_EPI;
    extern __shared__ __align__(1024) unsigned char smem[];
    FcCtrl* c = const_cast<FcCtrl*>(a.ctrl);
    if (c->bad) return;
    const int items = 2 * a.groups * a.nseg;
    if ((int)blockIdx.x >= items) return;
    unsigned char* res = smem;                                  // [RC_MAX][2][16 KB]
    unsigned char* stg = smem + RES_BYTES;                      // [NST][16 KB]
    uint64_t* rfull = reinterpret_cast<uint64_t*>(smem + RES_BYTES + NST * CHUNK_BYTES);
    uint64_t* rfree = rfull + RC_MAX;
    uint64_t* sfull = rfree + RC_MAX;
    uint64_t* sfree = sfull + NST;
    uint64_t* accf = sfree + NST;
    uint64_t* acce = accf + 2;
    uint64_t* drain = acce + 2;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
    float* sinv_all = reinterpret_cast<float*>(smem + RES_BYTES + NST * CHUNK_BYTES + 1024);
    const int tid = threadIdx.x, warp = tid >> 5;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int q = 0; q < RC_MAX; ++q) {
            mbar_init(&rfull[q], 1);
            mbar_init(&rfree[q], 1);
        }
        for (int q = 0; q < NST; ++q) {
            mbar_init(&sfull[q], 1);
            mbar_init(&sfree[q], 1);
        }
        mbar_init(&accf[0], 1);
        mbar_init(&accf[1], 1);
        mbar_init(&acce[0], EPI);
        mbar_init(&acce[1], EPI);
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
    const int nch = a.nchunks;
    bool failed = false;

    if (warp == EPI) {
        // ---------------------------------------------------------- bulk copies
        if ((tid & 31) == 0) {
            uint32_t rfree_ph[RC_MAX] = {0, 0, 0, 0}, sfree_ph[NST] = {0, 0, 0, 0, 0};
            int rloads = 0;                   // resident fills issued (one per item and bin)
            long long sloads = 0;             // streamed blocks issued
            long long scount[NST] = {0, 0, 0, 0, 0};
            for (int it = (int)blockIdx.x; it < items && !failed; it += (int)gridDim.x) {
                const ResItem I = res_item(a, it);
                const int kr = I.p == 0 ? 0 : 2;  // row side: XR, XI or UR, UI; column side: XR or UR
                for (int f = I.f0; f < I.f1 && !failed; ++f) {
                    for (int q = 0; q < nch; ++q) {
                        if (rloads > 0) {  // the MMAs of the previous bin have read this slot
                            if (!mbar_wait_bounded(&rfree[q], rfree_ph[q])) { failed = true; break; }
                            rfree_ph[q] ^= 1;
                        }
                        // the two kinds back to back, so that the second continues the first's
                        // 8-row groups (a 256-row operand); a short last chunk moves less
                        const uint32_t qb = (uint32_t)chunk_cols(a.last_kc, q, nch) * 2048u;
                        unsigned char* dst = res + (size_t)q * 2 * CHUNK_BYTES;
                        mbar_expect_tx(&rfull[q], 2 * qb);
                        bulk_g2s(dst, op_block(a, I.a, f, kr, q), qb, &rfull[q]);
                        bulk_g2s(dst + qb, op_block(a, I.a, f, kr + 1, q), qb, &rfull[q]);
                    }
                    if (failed) break;
                    ++rloads;
                    for (int b = I.b0; b < I.b1 && !failed; ++b)
                        for (int q = 0; q < nch; ++q) {
                            const int st = (int)(sloads % NST);
                            if (sloads >= NST) {
                                if (!mbar_wait_bounded(&sfree[st], sfree_ph[st])) { failed = true; break; }
                                sfree_ph[st] ^= 1;
                            }
                            const uint32_t qb = (uint32_t)chunk_cols(a.last_kc, q, nch) * 2048u;
                            mbar_expect_tx(&sfull[st], qb);
                            bulk_g2s(stg + (size_t)st * CHUNK_BYTES, op_block(a, b, f, kr, q), qb, &sfull[st]);
                            ++scount[st];
                            ++sloads;
                        }
                }
            }
            // let every copy issued land before the CTA ends
            if (rloads > 0)
                for (int q = 0; q < nch; ++q) mbar_wait_bounded(&rfull[q], (uint32_t)((rloads - 1) & 1));
            for (int st = 0; st < NST; ++st)
                if (scount[st] > 0) mbar_wait_bounded(&sfull[st], (uint32_t)((scount[st] - 1) & 1));
        }
    } else if (warp == EPI + 1) {
        // ---------------------------------------------------------- MMAs
        if ((tid & 31) == 0) {
            // N = 256: the row tile's two kinds (XR_a then XI_a, or UR_a then UI_a) are adjacent
            // in shared memory with the 8-row-group stride, so one MMA takes both as a
            // 256-row operand and writes both accumulators (TMEM columns 0-127 and 128-255)
            const uint32_t idesc = make_idesc(KIND == 1 ? 2u : (a.ab_format == 1 ? 1u : 0u), TILE, 2 * TILE);
            uint32_t rfull_ph[RC_MAX] = {0, 0, 0, 0}, sfull_ph[NST] = {0, 0, 0, 0, 0}, acce_ph[2] = {0, 0};
            long long sused = 0, u = 0;
            for (int it = (int)blockIdx.x; it < items && !failed; it += (int)gridDim.x) {
                const ResItem I = res_item(a, it);
                for (int f = I.f0; f < I.f1 && !failed; ++f)
                    for (int b = I.b0; b < I.b1 && !failed; ++b) {
                        const int buf = (int)(u & 1);
                        if (u >= 2) {  // the epilogue has drained this TMEM buffer
                            if (!mbar_wait_bounded(&acce[buf], acce_ph[buf])) { failed = true; break; }
                            acce_ph[buf] ^= 1;
                            fence_after();
                        }
                        const uint32_t d = tmem + (uint32_t)(buf * 2 * TILE);
                        for (int q = 0; q < nch; ++q) {
                            if (b == I.b0) {  // this bin's resident chunk has landed
                                if (!mbar_wait_bounded(&rfull[q], rfull_ph[q])) { failed = true; break; }
                                rfull_ph[q] ^= 1;
                            }
                            const int st = (int)(sused % NST);
                            if (!mbar_wait_bounded(&sfull[st], sfull_ph[st])) { failed = true; break; }
                            sfull_ph[st] ^= 1;
                            fence_after();
                            const uint32_t sb = smem_u32(stg + (size_t)st * CHUNK_BYTES);
                            const uint32_t r0 = smem_u32(res + (size_t)q * 2 * CHUNK_BYTES);
                            const int cols = chunk_cols(a.last_kc, q, nch);  // 2 per K-step
                            const uint32_t sbo = (uint32_t)cols * 128u;
#pragma unroll
                            for (int ks = 0; ks < 4; ++ks) {
                                if (2 * ks >= cols) break;
                                const uint32_t acc = (q > 0 || ks > 0) ? 1u : 0u;
                                const uint32_t off = ks * 256;
                                const uint64_t d_b = smem_desc_sbo(sb + off, sbo);          // XR_b or UR_b
                                const uint64_t d_a2 = smem_desc_sbo(r0 + off, sbo);         // [XR_a; XI_a] or [UR_a; UI_a]
                                mma<KIND>(d, d_b, d_a2, idesc, acc);
                            }
                            mma_commit(&sfree[st]);                 // the stage may be refilled
                            if (b == I.b1 - 1) mma_commit(&rfree[q]);  // last tile of the bin: slot free
                            ++sused;
                        }
                        if (failed) break;
                        mma_commit(&accf[buf]);
                        ++u;
                    }
            }
            mma_commit(drain);
            mbar_wait_bounded(drain, 0);
        }
    } else {
        // ---------------------------------------------------------- epilogue (warps 0 .. EPI-1)
        uint32_t accf_ph[2] = {0, 0};
        const int quarter = warp & 3, rpart = warp >> 2;  // TMEM lanes 32 quarter ..; rows RES_ROWS rpart ..
        const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
        float* sinv = sinv_all + warp * RES_ROWS;  // this warp's rows: no barrier across warps
        const int ibase = rpart * RES_ROWS;
        long long u = 0;
        // 1/sqrt(PSD) one step ahead: the next bin's row values of this warp (loaded during the
        // current bin) and the next unit's column value of this thread
        constexpr int RPL = RES_ROWS / 32;  // row values per lane
        float pf_row[RPL], pf_col = 0.f;
        auto load_row = [&](const ResItem& I, int f) {
#pragma unroll
            for (int r = 0; r < RPL; ++r) {
                const int i = I.a * TILE + ibase + 32 * r + (tid & 31);
                pf_row[r] = (I.p == 0 && i < a.n) ? a.inv_psd[(size_t)f * a.n + i] : 0.f;
            }
        };
        auto load_col = [&](const ResItem& I, int f, int tb) {
            const int jj = tb * TILE + quarter * 32 + (tid & 31);
            return (I.p == 0 && jj < a.n) ? a.inv_psd[(size_t)f * a.n + jj] : 0.f;
        };
        {
            const ResItem I0 = res_item(a, (int)blockIdx.x);
            load_row(I0, I0.f0);
            pf_col = load_col(I0, I0.f0, I0.b0);
        }
        for (int it = (int)blockIdx.x; it < items && !failed; it += (int)gridDim.x) {
            const ResItem I = res_item(a, it);
            const int ta = I.a;
            float* out = a.part + (size_t)I.g * 3 * a.P + (I.p == 0 ? 0 : 2 * a.P);  // this group's band sums
            for (int f = I.f0; f < I.f1 && !failed; ++f) {
                const bool first = f == I.f0;  // the group's first bin stores, later bins add
                __syncwarp();
#pragma unroll
                for (int r = 0; r < RPL; ++r) sinv[32 * r + (tid & 31)] = pf_row[r];
                __syncwarp();
                {  // the next bin of this item, or the first bin of the next item
                    const int itn = f + 1 < I.f1 ? it : it + (int)gridDim.x;
                    if (itn < items) {
                        const ResItem In = itn == it ? I : res_item(a, itn);
                        load_row(In, itn == it ? f + 1 : In.f0);
                    }
                }
                for (int tb = I.b0; tb < I.b1; ++tb) {
                    const int buf = (int)(u & 1);
                    const int j = tb * TILE + quarter * 32 + (tid & 31);  // this thread's TMEM lane: column node j
                    const float inv_j = pf_col;
                    {  // the next unit's column value
                        int nit = it, nf = f, ntb = tb + 1;
                        if (ntb >= I.b1) { ntb = I.b0; ++nf; }
                        if (nf >= I.f1) nit = it + (int)gridDim.x;
                        if (nit < items) {
                            const ResItem In = nit == it ? I : res_item(a, nit);
                            if (nit != it) { nf = In.f0; ntb = In.b0; }
                            pf_col = load_col(In, nf, ntb);
                        }
                    }
                    const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(&accf[buf], accf_ph[buf]) ? 1 : 0) != 0;
                    accf_ph[buf] ^= 1;
                    if (!ok) {
                        failed = true;
                        break;
                    }
                    fence_after();
                    const uint32_t col = (uint32_t)(buf * 2 * TILE);
                    // this warp's RES_ROWS rows in two halves of NG groups of 16 TMEM columns (the
                    // register file, split over the four schedulers, allows ~170 registers here)
                    constexpr int NG = RES_ROWS / 32;
#pragma unroll 1
                    for (int hh = 0; hh < 2; ++hh) {
                    const int hbase = ibase + hh * (RES_ROWS / 2);
                    uint32_t rre[NG][16], rim[NG][16];
#pragma unroll
                    for (int s4 = 0; s4 < NG; ++s4) {
                        tmem_ld16_issue(lane_base + col + hbase + 16 * s4, rre[s4]);
                        tmem_ld16_issue(lane_base + col + TILE + hbase + 16 * s4, rim[s4]);
                    }
                    tmem_wait_ld();
#pragma unroll
                    for (int s4 = 0; s4 < NG; ++s4) {
                        tmem_keep(rre[s4]);
                        tmem_keep(rim[s4]);
                    }
                    if (j < a.n) {
                        // as in k_herk_tc: packed index p(i + 1) = p(i) + n - i - 2; off-diagonal tile
                        // pairs (ta < tb) need no per-element test
                        auto emit = [&](auto first_c, auto full_c, auto phase_c) {
                            constexpr bool FIRST = decltype(first_c)::value;
                            constexpr bool FULL = decltype(full_c)::value;
                            constexpr int PH = decltype(phase_c)::value;
                            int i = ta * TILE + hbase;
                            int pk = (int)packed_index(i, j, a.n);
                            float* out2 = out + a.P;  // IMAGCOHY plane (phase A)
                            const float2 invj2 = make_float2(inv_j, inv_j);
                            // one value per element: the first bin stores, later bins reduce
                            auto put = [&](float* base, int at, float v) {
                                if (FIRST) base[at] = v;
                                else atomicAdd(base + at, v);
                            };
#pragma unroll
                            for (int s4 = 0; s4 < NG; ++s4) {
#pragma unroll
                                for (int q = 0; q < 16; q += 2) {
                                    // two row nodes i, i + 1 per packed FP32x2 operation
                                    const float2 vre = make_float2(__uint_as_float(rre[s4][q]), __uint_as_float(rre[s4][q + 1]));
                                    const float2 vim = make_float2(__uint_as_float(rim[s4][q]), __uint_as_float(rim[s4][q + 1]));
                                    float2 v0, v1;
                                    if (PH == 0) {
                                        const float2 sc = mul2(*reinterpret_cast<const float2*>(&sinv[hh * (RES_ROWS / 2) + 16 * s4 + q]), invj2);
                                        const float2 r = mul2(vre, sc), m = mul2(vim, sc);
                                        const float2 t = fma2(r, r, mul2(m, m));
                                        v0 = make_float2(sqrt_approx(t.x), sqrt_approx(t.y));
                                        v1 = m;
                                    } else {
                                        const float2 t = fma2(vre, vre, mul2(vim, vim));
                                        v0 = make_float2(__fmul_rn(sqrt_approx(t.x), inv_K), __fmul_rn(sqrt_approx(t.y), inv_K));
                                        v1 = v0;
                                    }
#pragma unroll
                                    for (int e = 0; e < 2; ++e, pk += a.n - i - 2, ++i) {
                                        if (!FULL && (j <= i || i >= a.n)) continue;
                                        put(out, pk, e ? v0.y : v0.x);
                                        if (PH == 0) put(out2, pk, e ? v1.y : v1.x);
                                    }
                                }
                            }
                        };
                        const bool full = ta < tb;
                        using T = std::true_type;
                        using F = std::false_type;
                        using P0 = std::integral_constant<int, 0>;
                        using P1 = std::integral_constant<int, 1>;
                        if (I.p == 0) {
                            if (first) { if (full) emit(T{}, T{}, P0{}); else emit(T{}, F{}, P0{}); }
                            else { if (full) emit(F{}, T{}, P0{}); else emit(F{}, F{}, P0{}); }
                        } else {
                            if (first) { if (full) emit(T{}, T{}, P1{}); else emit(T{}, F{}, P1{}); }
                            else { if (full) emit(F{}, T{}, P1{}); else emit(F{}, F{}, P1{}); }
                        }
                    }
                    }  // halves
                    fence_before();
                    __syncwarp();
                    if ((tid & 31) == 0)
                        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acce[buf])) : "memory");
                    ++u;
                }
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

__device__ __forceinline__ uint32_t tf32_bits(float x) {
    uint32_t t;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(t) : "f"(x));
    return t;
}
// Split TF32: x = hi + lo with hi = tf32(x) and lo = tf32(x - hi) (x - hi is exact in FP32).
__device__ __forceinline__ float tf32_low(float x) { return __fsub_rn(x, __uint_as_float(tf32_bits(x))); }

// low = true: the low parts of a split-TF32 operand (ab_format 3).
__device__ __forceinline__ uint4 pack_chunk(const float (&v)[8], int per16, int ab_format, bool low = false) {
    if (ab_format >= 2) {  // TF32: round to nearest (ties away), stored in 32-bit words
        uint32_t t[4];
        for (int q = 0; q < 4; ++q) t[q] = tf32_bits(low ? tf32_low(v[q]) : v[q]);
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
    const int slot0 = (int)(start % a.slots);  // ring slot of the window's first trial
    const int esize = a.ab_format >= 2 ? 4 : 2;
    const int per16 = 16 / esize;                 // elements per 16-byte unit
    // unit e = (block index (tile, bin, chunk)) * 1024 + (m8 * 8 + kc) * 8 + r: the low ten
    // bits give the place in the block, the block index is split with 32-bit arithmetic
    const long long total = (long long)a.ntiles * a.B * a.nchunks * 1024;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        const unsigned low = (unsigned)e & 1023u;
        const int r = (int)(low & 7u), kc = (int)((low >> 3) & 7u), m8 = (int)(low >> 6);
        const unsigned blk = (unsigned)(e >> 10);
        const int ch = (int)(blk % (unsigned)a.nchunks);
        const unsigned tf = blk / (unsigned)a.nchunks;
        const int f = (int)(tf % (unsigned)a.B), tile = (int)(tf / (unsigned)a.B);
        const int cols = chunk_cols(a.last_kc, ch, a.nchunks);
        if (kc >= cols) continue;  // not stored (zero padding of a short last chunk)
        const int m = m8 * 8 + r;
        const int node = tile * TILE + m;
        const int k0 = (ch * 8 + kc) * per16;           // first inner index of this 16-byte unit
        const float2* col = a.ring + (size_t)f * a.n + node;
        const size_t slot_stride = (size_t)a.B * a.n;
        float v[4][8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int k = k0 + q;
            v[0][q] = v[1][q] = v[2][q] = v[3][q] = 0.f;  // padding: +0 exactly
            bool take = false;
            int slot = 0, part = 0;
            if (a.ring_order) {  // position k: slot k (first half) or k - slots (second half)
                part = k >= a.slots;
                slot = part ? k - a.slots : k;
                if (slot < a.slots) {  // the window's trial in this slot, if any
                    const long long t = end - 1 - (((end - 1 - slot) % a.slots) + a.slots) % a.slots;
                    take = t >= start && t >= 0;
                }
            } else if (k < 2 * K) {
                part = k >= K;
                slot = slot0 + (part ? k - K : k);
                if (slot >= a.slots) slot -= a.slots;
                take = true;
            }
            if (q < per16 && node < a.n && take) {
                const float2 X = col[(size_t)slot * slot_stride];
                const float2 u = phasor_of_x(X);
                v[0][q] = part ? X.y : X.x;   // XR
                v[1][q] = part ? -X.x : X.y;  // XI
                v[2][q] = part ? u.y : u.x;   // UR
                v[3][q] = part ? -u.x : u.y;  // UI
            }
        }
        const int nk = op_kinds(a.ab_format);
#pragma unroll
        for (int kind = 0; kind < 8; ++kind) {
            if (kind >= nk) break;
            unsigned char* dst = a.ops + ((((size_t)tile * a.B + f) * nk + kind) * a.nchunks + ch) * (size_t)CHUNK_BYTES +
                                 (size_t)((m8 * cols + kc) * 8 + r) * 16;
            *reinterpret_cast<uint4*>(dst) = pack_chunk(v[kind & 3], per16, a.ab_format, kind >= 4);
        }
    }
}

// Operand ring of a mixed-precision streaming session. Element (tile row m, inner k) of the
// block (tile, bin, kind, chunk) as in k_pack_operands, with the ring slot s of a trial at
// inner positions s (first half) and slots + s (second half). One thread per (slot entry,
// bin, node) writes that element of all four kinds; slots outside the window hold zeros.
__device__ __forceinline__ void put_elem(unsigned char* ops, const PackArgs& a, int tile, int f, int kind, int m,
                                         int k, float v) {
    const int esize = a.ab_format >= 2 ? 4 : 2;
    const int per16 = 16 / esize;
    const int chunk = k / (8 * per16), kc = (k / per16) % 8, e16 = k % per16;
    const int cols = chunk_cols(a.last_kc, chunk, a.nchunks);  // kc < cols for every stored k
    const int nk = op_kinds(a.ab_format);
    unsigned char* dst = ops + ((((size_t)tile * a.B + f) * nk + kind) * a.nchunks + chunk) * (size_t)CHUNK_BYTES +
                         (size_t)((m / 8) * cols + kc) * 128 + (m % 8) * 16 + e16 * esize;
    if (a.ab_format == 3) {  // split TF32: the high part here, the low part in kind + 4
        *reinterpret_cast<uint32_t*>(dst) = tf32_bits(v);
        unsigned char* dl = dst + (size_t)4 * a.nchunks * CHUNK_BYTES;
        *reinterpret_cast<uint32_t*>(dl) = tf32_bits(tf32_low(v));
    } else if (a.ab_format == 2) {
        *reinterpret_cast<uint32_t*>(dst) = tf32_bits(v);
    } else if (a.ab_format == 1) {
        *reinterpret_cast<__nv_bfloat16*>(dst) = __float2bfloat16_rn(v);
    } else {
        *reinterpret_cast<__half*>(dst) = __float2half_rn(v);
    }
}

__global__ void k_pack_ring(PackArgs a, int mode) {
    const FcCtrl* c = a.ctrl;
    if (c->bad) return;
    const long long end = c->pushed + a.count;  // window after this call: [end - W, end)
    const long long start = end > a.W ? end - a.W : 0;
    // mode 0: the newest slot written, the next one (whose trial left) cleared; mode 1: every
    // slot from the window; mode 2: the newest slot only (full mode: W slots, so the newest
    // trial's slot is the one whose trial left)
    const int nslot = mode == 0 ? 2 : (mode == 2 ? 1 : a.slots);
    const long long total = (long long)nslot * a.B * a.n;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        const int node = (int)(e % a.n);
        const int f = (int)((e / a.n) % a.B);
        const int q = (int)(e / ((long long)a.n * a.B));
        // mode 0: q = 0 the newest trial's slot, q = 1 the slot of the trial that left
        const int s = mode != 1 ? (int)((q == 0 ? end - 1 : end) % a.slots) : q;
        bool in_window = false;
        if (mode != 1) {
            in_window = q == 0;
        } else {
            // the window's trial in slot s, if any: t = s (mod slots), start <= t < end
            const long long t = end - 1 - (((end - 1 - s) % a.slots) + a.slots) % a.slots;
            in_window = t >= start && t >= 0;
        }
        float2 X = make_float2(0.f, 0.f);
        if (in_window) X = a.ring[((size_t)s * a.B + f) * a.n + node];
        const float2 u = phasor_of_x(X);
        const int tile = node / TILE, m = node % TILE;
        const float v[2][4] = {{X.x, X.y, u.x, u.y}, {X.y, -X.x, u.y, -u.x}};
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int kind = 0; kind < 4; ++kind) put_elem(a.ops, a, tile, f, kind, m, h * a.slots + s, v[h][kind]);
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
    cudaError_t e;
    if (a.seg_a && a.nchunks <= RC_MAX) {  // resident-operand form (never split TF32)
        if (a.ab_format == 3) return cudaErrorInvalidValue;
        const int items = 2 * a.groups * a.nseg;
        const int ctas = items < a.grid_ctas ? items : a.grid_ctas;
        if (a.ab_format == 2) {
            e = cudaFuncSetAttribute(k_herk_res<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, RES_SMEM);
            if (e != cudaSuccess) return e;
            k_herk_res<1><<<ctas, RES_THREADS, RES_SMEM, st>>>(a);
        } else {
            e = cudaFuncSetAttribute(k_herk_res<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, RES_SMEM);
            if (e != cudaSuccess) return e;
            k_herk_res<0><<<ctas, RES_THREADS, RES_SMEM, st>>>(a);
        }
        return cudaGetLastError();
    }
    // the streaming-operand form reads full chunks only
    if (a.last_kc >= 2 && a.last_kc < 8) return cudaErrorInvalidValue;
    const int units = a.ntp * a.groups;
    const int ctas = units < a.grid_ctas ? units : a.grid_ctas;
    if (a.ab_format == 3) {
        constexpr int sm = HerkStages<true>::SMEM;
        e = cudaFuncSetAttribute(k_herk_tc<1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        if (e != cudaSuccess) return e;
        k_herk_tc<1, true><<<ctas, THREADS, sm, st>>>(a);
    } else if (a.ab_format == 2) {
        constexpr int sm = HerkStages<false>::SMEM;
        e = cudaFuncSetAttribute(k_herk_tc<1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        if (e != cudaSuccess) return e;
        k_herk_tc<1, false><<<ctas, THREADS, sm, st>>>(a);
    } else {
        constexpr int sm = HerkStages<false>::SMEM;
        e = cudaFuncSetAttribute(k_herk_tc<0, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        if (e != cudaSuccess) return e;
        k_herk_tc<0, false><<<ctas, THREADS, sm, st>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_pack_ring(const PackArgs& a, int mode, cudaStream_t st) {
    const long long total = (long long)(mode == 0 ? 2 : (mode == 2 ? 1 : a.slots)) * a.B * a.n;
    long long blocks = (total + 255) / 256;
    const long long cap = 8LL * fc_device_sms();
    if (blocks > cap) blocks = cap;
    k_pack_ring<<<(unsigned)(blocks < 1 ? 1 : blocks), 256, 0, st>>>(a, mode);
    return cudaGetLastError();
}

cudaError_t launch_herk_band(const HerkArgs& a, cudaStream_t st) {
    k_herk_band<<<(unsigned)((a.P + 255) / 256), 256, 0, st>>>(a);
    return cudaGetLastError();
}

size_t herk_chunk_bytes() { return CHUNK_BYTES; }
int herk_resident_max_chunks() { return RC_MAX; }
