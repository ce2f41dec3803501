// fc_internal.h - session state, device layout and kernel launchers (library-internal).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/fc.h"

// ---------------------------------------------------------------------------------
// Device layout
//
// Nodes are grouped in tiles of FC_T = 32. The pair space is covered by the upper
// triangle of tile pairs (a <= b), enumerated row by row; a diagonal tile pair (a == a)
// holds only its pairs with i < j.
//
// Spectral accumulators, one block per (tile pair, bin), tile-pair major, bins inside:
//   block = 13 planes of FC_T*FC_T 32-bit words, pair (li, lj) at word li*32 + lj:
//     planes 2k, 2k+1 = hi, lo floats of double-float field k:
//       k = 0 CSD re, 1 CSD im (= sum Im, also used by WPLI/DSWPLI), 2 phasor re,
//           3 phasor im, 4 sum |Im|, 5 sum Im^2
//     plane 12      = int32 sign count
//   53,248 bytes per (tile pair, bin): 52 B per pair-bin of state.
// Ring of spectra: slots x [n_bins][n_nodes] float2 (re, im), a slot per stored trial.
// Per-node: psd [n_bins][n_nodes] double; inv_sqrt_psd [n_bins][n_nodes] float.
// Networks: [FC_NMETRIC][P] float, packed upper (pair (i,j), i<j).
// Time-domain accumulators (COR, XCOR): double-float [2][P] (hi plane, lo plane).
// ---------------------------------------------------------------------------------

#define FC_T 32
#define FC_TT (FC_T * FC_T)
#define FC_NFIELD 6
#define FC_BLOCK_WORDS (13 * FC_TT)
#define FC_NMETRIC 9

// metric bit index (log2 of the FC_* bit)
enum { MI_COR = 0, MI_XCOR, MI_COH, MI_IMAGCOHY, MI_PLV, MI_PLI, MI_USPLI, MI_WPLI, MI_DSWPLI };

// Device-resident control block: the state of the window lives on the device so that a
// push never waits for the host (rejections are decided on the device).
struct FcCtrl {
    long long pushed;      // accepted trials
    long long rejected;    // rejected trials
    int bad;               // the push in flight held a non-finite value
    int bad_latched;       // a rejection happened since the host last looked
    unsigned int max_bits; // calibration: max |re|,|im| of the first spectra (float bits)
    float scale;           // power-of-two prescale of all spectra (0 = not calibrated)
    int timeout;           // a bounded device-side wait ran out
    float in_scale;        // power-of-two factor the full-window kernels apply to the spectra
                           // as they read them (0: none; sessions store prescaled spectra)
};

struct FcPendingTiming {
    int kernel;
    cudaEvent_t start, stop;
};

struct fc_session {
    // settings
    int n, N, B, first_bin, nfft, W, slots;
    double fs;
    fc_band band;
    fc_taper taper;
    uint32_t mask;      // metrics finalized each push
    uint32_t time_mask; // COR/XCOR state allocated at creation
    bool spectral;      // spectral state (spectra ring, pair sums) allocated at creation
    fc_config cfg;
    bool own_stream;
    cudaStream_t stream;
    int device;
    int num_sms;

    // derived sizes
    int nt;             // node tiles
    int ntp;            // tile pairs
    long long P;        // pairs
    int groups;         // bin groups for the full-window kernel
    int group_bins;     // bins per group
    int stream_groups;  // bin groups for the streaming kernel
    int stream_group_bins;
    int xcor_L;         // XCOR transform length (power of two >= 2N - 1)

    // host mirror of the enqueued push count (scheduling only; the device count rules)
    long long enqueued;
    long long resum_phase;  // next slice of the sliced re-sum (0 .. period - 1)
    bool calibrated;        // the device prescale is known to be set
    int sel0, sel1;         // selected sub-band: bins sel0 .. sel1 - 1 of the B computed

    float* dense_scratch;   // n x n staging for dense host outputs
    size_t dense_scratch_len;
    void* post_scratch;     // network post-processing: select state, ties, flags, outputs
    size_t post_scratch_len;
    float* cor_part;        // COR full-window trial-group partial sums (allocated on demand)
    size_t cor_part_len;
    float* proj;            // source projection M [n][proj_C] (NULL: none)
    int proj_C;
    float* proj_in;         // staged sensor trials [proj_in_trials][proj_C][N]
    int proj_in_trials;
    bool spec_project;      // this push projects band spectra (a projection and no COR / XCOR)
    float2* sens_spec;      // sensor band spectra of the trials of one push [sens_trials][B][proj_C]
    int sens_trials;

    // device buffers
    FcCtrl* ctrl;
    float* x_stage;         // [stage_trials][n][N]
    int stage_trials;
    float2* twiddle;        // [N][B] taper-folded DFT factors (DFT spectrum method)
    bool use_fft;           // spectrum by real FFT instead of the band DFT
    float* taper_tab;       // FFT method: [N] taper
    float2* fft_tw;         // FFT method: [nfft/2] twiddles e^{-2 pi i k / nfft}
    float2* ring;           // [slots][B][n]
    double* psd;            // [B][n]
    float* inv_psd;         // [B][n]
    float* acc;             // [ntp][B][13][1024] (stream mode)
    unsigned short* tile_a; // [ntp]
    unsigned short* tile_b; // [ntp]
    float* net;             // [FC_NMETRIC][P]
    float* partial;         // [groups][7][P] band partial sums (when groups > 1)
    int partial_groups;     // bin groups the partial planes are allocated for
    float* zring;           // COR: [slots][n][N] normalized trials
    float* cor_acc;         // COR: [2][P] double-float
    float* xcor_vals;       // XCOR: [slots][P] per-trial values
    int* xcor_lag;          // XCOR: [P] lags of the newest trial
    float* xcor_acc;        // XCOR: [2][P]
    float2* xcor_tw;        // XCOR FFT twiddles [L/2]
    float2* xcor_spec;      // XCOR spectra of the trials in flight [count][n][L/2+1]
    float* xcor_energy;     // XCOR [count][n]
    int xcor_spec_trials;
    // tensor-core full-window path (precision BF16 / FP16 / TF32)
    int nt128, ntp128, nchunks, ab_format;
    int last_kc = 8;        // core-matrix columns of the last operand K-chunk (see PackArgs)
    unsigned short* tile_a128;
    unsigned short* tile_b128;
    unsigned char* ops;     // packed operands [nt128][B][4 kinds, 8 for split TF32][nchunks][16 KB]
    unsigned char* tiny_flags;  // [B][n] a trial of the window has a tiny component (mixed path)
    bool mixed_stream;      // streaming session whose re-sum takes the linear sums from the tensor cores
    int* list32;            // mixed streaming: 32-node tile pairs grouped by 128-node tile pair
    std::vector<int> list32_off;  // (host) first list entry of each 128-node tile pair, [ntp128 + 1]
    unsigned char* cor_ops; // COR split-TF32 operand ring [slots][cor_nt][cor_nchunks][2][16 KB]
    int cor_nt, cor_ntp, cor_nchunks;
    unsigned short* seg_a;  // resident-operand segments of the 128-node tile pairs (see HerkArgs)
    unsigned short* seg_b0;
    unsigned short* seg_b1;
    int nseg, seg_max;
    float* herk_part;       // [herk_gcap][3][P] band sums of COH, IMAGCOHY, PLV per bin group
    int herk_gcap;          // bin groups the band-sum planes are allocated for
    size_t device_bytes;

    // measurement
    long long launches;
    bool profiling;
    std::vector<FcPendingTiming> pending;
    fc_kernel_time ktime[FC_K_COUNT];
    std::vector<void*> allocations;
    std::vector<std::pair<void*, size_t>> state_bufs;  // persistent state, in allocation order

    // pipelined host I/O (created on first use): single host trials are copied in on
    // in_stream into alternating buffers; async network reads leave on out_stream from a
    // device snapshot of the plane
    cudaStream_t in_stream = nullptr, out_stream = nullptr;
    // drift re-sum overlapped with the streaming update: the slice of a push (FP32 sessions:
    // the whole exact re-sum; mixed-precision sessions: its non-linear sums) runs on
    // side_stream (lowest priority) into resum_scratch (resum_scratch_tp 32-node tile pairs x
    // all bins) beside k_stream; the scratch goes over the slice's accumulator blocks (their
    // non-linear planes for mixed precision) once both are done
    float* resum_scratch = nullptr;
    int resum_scratch_tp = 0;
    cudaStream_t side_stream = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // a batched (served) push's slice: tile pairs resum_tp0 .. resum_tp1 - 1, forked after the
    // push's per-node sums, copied in when its last share of the update is done
    int resum_tp0 = 0, resum_tp1 = 0;
    bool resum_pending = false, resum_forked = false;
    float* x_in[2] = {nullptr, nullptr};
    cudaEvent_t ev_in[2] = {nullptr, nullptr};    // the copy into x_in[b] has landed
    cudaEvent_t ev_used[2] = {nullptr, nullptr};  // the push that read x_in[b] is done
    bool used_valid[2] = {false, false};
    int in_flip = 0;
    float* snap[2] = {nullptr, nullptr};          // [P] each
    cudaEvent_t ev_snap[2] = {nullptr, nullptr};  // snapshot b taken (compute stream)
    cudaEvent_t ev_out[2] = {nullptr, nullptr};   // snapshot b landed in host memory
    int out_head = 0, out_count = 0;
};

// ---------------------------------------------------------------------------------
// Launchers (each returns the cudaError_t of the launch)

struct SpectrumArgs {
    const float* x;        // [count][n][N]
    int count;             // trials in x
    int write_from;        // first trial of x written to the ring (earlier ones are skipped)
    const float2* twiddle; // [N][B]
    float2* ring;
    int slots, n, N, B;
    FcCtrl* ctrl;
    int direct;            // 1: trial write_from + t into slot t of `ring`, unscaled (sensor spectra)
    // real-FFT method (fft = 1): taper [N], twiddles [nfft/2], band bins first_bin .. + B - 1;
    // the radices of nfft/2, four bits per pass, first pass in the low bits
    int fft, nfft, first_bin, fft_stages;
    unsigned long long fft_radices;
    const float* taper;
    const float2* fft_tw;
};
cudaError_t launch_validate(const float* x, long long count, FcCtrl* ctrl, cudaStream_t st);
cudaError_t launch_spectrum(const SpectrumArgs& a, cudaStream_t st);
cudaError_t launch_calibrate(const SpectrumArgs& a, cudaStream_t st, int phase);

struct NodeArgs {
    const float2* ring;
    double* psd;
    float* inv_psd;
    int slots, n, B, W;
    int mode;   // 0 = add newest / subtract leaving, 1 = recompute from the window
    FcCtrl* ctrl;
    int count;  // trials pushed by this call (mode 1: the window ends at pushed + count)
    unsigned char* tiny;  // optional [B][n] tiny-component flags: mode 1 sets them for the window's
                          // trials, mode 0 adds the new trial's (flags of leaving trials stay set)
};
cudaError_t launch_node(const NodeArgs& a, cudaStream_t st);

struct PairArgs {
    const float2* ring;
    const float* inv_psd;
    float* acc;
    const unsigned short* tile_a;
    const unsigned short* tile_b;
    float* net_spec;   // network planes of the 7 spectral metrics, [7][P] (COH .. DSWPLI)
    float* partial;    // [groups][7][P]
    int slots, n, B, W, ntp;
    long long P;
    int groups, group_bins;
    uint32_t mask;     // metrics to finalize
    int finalize;      // write networks / partials
    int update;        // stream kernel: 1 = add/subtract the trials, 0 = finalize only
    int write_acc;     // window kernel: store accumulators (re-sum)
    int tp0, tp_count; // window kernel: tile pairs tp0 .. tp0 + tp_count - 1 (tp_count 0: all)
    int acc_tp_base;   // window kernel: the accumulator block of tile pair tp is acc[tp - acc_tp_base]
    int acc_by_pos;    // non-linear re-sum: block i of the list goes to acc[i] (a scratch), not acc[tp]
    int u0;            // stream kernel: first unit of this launch (a push may span launches)
    int fsel0, fsel1;  // bins fsel0 .. fsel1 - 1 enter the band average (a sub-band of the B)
    int count;         // trials pushed by this call (window end = pushed + count)
    int grid_ctas;     // persistent grid size of the streaming kernel
    const FcCtrl* ctrl;
    const unsigned char* tiny;  // non-linear sums: [B][n] tiny-component flags of the window (k_node)
    const int* tp_list;         // non-linear re-sum: tile pairs tp_list[tp0 .. tp0 + tp_count - 1]
};
// The non-linear sums kernel storing its window sums (sum Im, sum |Im|, sum Im^2, sign count)
// into the accumulators of tile pairs tp_list[tp0 .. tp0 + tp_count - 1] (the linear fields
// are left as they are): the re-sum of a mixed-precision streaming session.
cudaError_t launch_nonlinear_acc(const PairArgs& a, cudaStream_t st);
cudaError_t launch_stream_update(const PairArgs& a, cudaStream_t st);

// A batch of sessions updated by one launch of the streaming kernel (passed by value as
// the kernel's parameter block). The launch covers units a[s].u0 .. a[s].u0 + (unit_prefix[s+1]
// - unit_prefix[s]) - 1 of session s; a session's push may be split over several launches.
#define FC_MAX_BATCH 32
struct StreamBatch {
    int nsess;
    int unit_prefix[FC_MAX_BATCH + 1];
    PairArgs a[FC_MAX_BATCH];
};
cudaError_t launch_stream_batch(const StreamBatch& b, int grid_ctas, cudaStream_t st);
cudaError_t launch_window_sums(const PairArgs& a, cudaStream_t st);
// nfloats (a multiple of 4) from src to dst, skipped when ctrl->bad (a rejected push)
cudaError_t launch_copy_blocks(const float* src, float* dst, long long nfloats, const FcCtrl* ctrl, cudaStream_t st);
// The non-linear planes (sum Im, sum |Im|, sum Im^2, sign count) of scratch block set i (B bins)
// into the accumulator blocks of tile pair list[i], i < count; skipped when ctrl->bad.
cudaError_t launch_gather_nonlinear(const float* scratch, float* acc, const int* list, int count, int B,
                                    const FcCtrl* ctrl, cudaStream_t st);
cudaError_t launch_band_reduce(const PairArgs& a, cudaStream_t st);
cudaError_t launch_bins_from_acc(const PairArgs& a, int metric_index, float* out, cudaStream_t st);
cudaError_t launch_bins_window(const PairArgs& a, int metric_index, float* out, cudaStream_t st);

// Tensor-core full-window linear sums (k_herk_tc.cu).
struct PackArgs {
    const float2* ring;
    unsigned char* ops;   // [tiles128][B][4 kinds, 8 for split TF32 (ab_format 3)][nchunks][16 KB]
    int n, B, W, slots, ntiles, nchunks, count;
    int ab_format;        // 0 = FP16, 1 = BF16, 2 = TF32, 3 = split TF32 (high + low parts)
    const FcCtrl* ctrl;
    int ring_order;       // full pack: inner positions by ring slot (s, slots + s) instead of by
                          // window order (k, K + k); slots outside the window hold zeros
    int last_kc;          // 16-byte core-matrix columns stored in the last K-chunk (2 .. 7: the
                          // short layout read by the resident-operand products; else all 8)
};
struct HerkArgs {
    const unsigned char* ops;
    const unsigned short* tile_a;  // 128-node tile pairs
    const unsigned short* tile_b;
    const float* inv_psd;
    float* part;          // [groups][3][P] band sums of COH, IMAGCOHY, PLV per bin group
    float* net;           // [FC_NMETRIC][P]
    int n, B, ntp, nchunks, W, count, ab_format, grid_ctas;
    int groups, group_bins;  // the selected bins in groups of group_bins (the last may be shorter)
    long long P;
    uint32_t mask;
    int fsel0, fsel1;     // bins entering the band average
    const FcCtrl* ctrl;
    // resident-operand form (nchunks <= 4): segments s = (row tile seg_a[s], column tiles
    // seg_b0[s] .. seg_b1[s] - 1); work items = 2 phases x groups x nseg
    const unsigned short* seg_a;
    const unsigned short* seg_b0;
    const unsigned short* seg_b1;
    int nseg, seg_max;
    int last_kc;          // as PackArgs::last_kc (the resident-operand form only)
    // accumulator mode (drift re-sum of a mixed-precision streaming session): the products of
    // 128-node tile pairs tp0 .. tp0 + ntp - 1 are written as the linear sums (CSD re, phasor
    // re and im) of the streaming accumulators acc (nt32 node tiles of 32), not as metrics
    float* acc_out;
    int tp0, nt32;
};
cudaError_t launch_pack_operands(const PackArgs& a, cudaStream_t st);
// Operand ring of a mixed-precision streaming session (inner position k < slots: ring slot k,
// first half; slots <= k < 2 slots: second half; slots outside the window hold zeros).
// mode 0: the newest trial's slot is written and the slot of the trial leaving the window
// cleared; mode 1: every slot rebuilt from the window (after a bulk push).
cudaError_t launch_pack_ring(const PackArgs& a, int mode, cudaStream_t st);
cudaError_t launch_herk_tc(const HerkArgs& a, cudaStream_t st);
cudaError_t launch_herk_band(const HerkArgs& a, cudaStream_t st);
size_t herk_chunk_bytes();
int herk_resident_max_chunks();
// Non-linear sums only (signs, |Im|, Im, Im^2) with the PLI/USPLI/WPLI/DSWPLI finalize.
// Bin groups partition the selected bins fsel0 .. fsel1 - 1 (group_bins each).
cudaError_t launch_nonlinear_sums(const PairArgs& a, cudaStream_t st);
int nonlinear_ctas_per_sm();

struct CommitArgs {
    FcCtrl* ctrl;
    int count;
};
cudaError_t launch_commit(const CommitArgs& a, cudaStream_t st);

// Several sessions' one-trial pushes in one launch per stage (serving): validation,
// spectrum and per-node sums of up to FC_MAX_BATCH sessions; the sessions' elements / CTAs
// follow each other (prefix sums), the work per session is that of the single kernels.
struct PreBatch {
    int nsess;
    long long val_prefix[FC_MAX_BATCH + 1];  // trial samples to validate
    int spec_prefix[FC_MAX_BATCH + 1];       // spectrum CTAs (32 nodes x 32 bins each)
    int node_prefix[FC_MAX_BATCH + 1];       // node-bin elements
    SpectrumArgs sp[FC_MAX_BATCH];
    NodeArgs nd[FC_MAX_BATCH];
};
cudaError_t launch_validate_batch(const PreBatch& b, cudaStream_t st);
cudaError_t launch_spectrum_batch(const PreBatch& b, cudaStream_t st);
cudaError_t launch_node_batch(const PreBatch& b, cudaStream_t st);
// Commit of several sessions' one-trial pushes; snap[s] (host memory reachable from the
// device, may be NULL) receives session s's control block after its commit.
struct CommitBatch {
    int nsess;
    FcCtrl* ctrl[FC_MAX_BATCH];
    FcCtrl* snap[FC_MAX_BATCH];
};
cudaError_t launch_commit_batch(const CommitBatch& b, cudaStream_t st);

// time-domain metrics
struct CorArgs {
    const float* x;     // [count][n][N] raw trials
    int count, write_from;
    float* zring;       // [slots][n][N]
    float* cor_acc;     // [2][P]
    float* net;         // network plane for COR
    int slots, n, N, W;
    long long P;
    int mode;           // 0 = stream add/subtract, 1 = full recompute of the window
    int finalize;
    int groups;         // mode 1: the window's trials split over this many CTAs per tile pair
    float* part;        // groups > 1: per-group double-float sums [groups][2][P]
    const FcCtrl* ctrl;
};
cudaError_t launch_cor_normalize(const CorArgs& a, cudaStream_t st);

// COR on the tensor cores (k_cor_tc.cu): split-TF32 operand ring and per-trial products.
struct CorTcArgs {
    const float* zring;       // [slots][n][N] normalized trials (pack input)
    unsigned char* ops;       // [slots][nt][nchunks][hi, lo][16 KB] TF32 operand blocks
    int n, N, nt, ntp, nchunks, slots, W;
    long long P;
    int count, write_from;    // this call's trials; the window ends at pushed + count
    int mode;                 // 0 = stream: add the newest trial, subtract the leaving one; 1 = window
    int groups;               // mode 1: the window's trials split over this many groups per tile pair
    float* cor_acc;           // [2][P] double-float sums
    float* net;               // COR plane
    float* part;              // groups > 1: [groups][2][P]
    int finalize;
    int grid_ctas;
    const FcCtrl* ctrl;
};
cudaError_t launch_cor_tc_pack(const CorTcArgs& a, cudaStream_t st);
cudaError_t launch_cor_tc(const CorTcArgs& a, cudaStream_t st);
size_t cor_tc_pair_bytes();
cudaError_t launch_cor_combine(const CorArgs& a, cudaStream_t st);

struct XcorArgs {
    const float* x;     // [count][n][N]
    int count, write_from;
    int n, N, L, W, slots;
    long long P;
    const float2* tw;   // [L/2] twiddles e^{-2 pi i k / L}
    float2* spec;       // [count][n][L/2+1]
    float* energy;      // [count][n]
    float* vals;        // [slots][P]
    int* lag;           // [P]
    float* acc;         // [2][P]
    float* net;
    int mode, finalize;
    const FcCtrl* ctrl;
};
cudaError_t launch_xcor_spectra(const XcorArgs& a, cudaStream_t st);
cudaError_t launch_xcor_pairs(const XcorArgs& a, cudaStream_t st);
cudaError_t launch_xcor_update(const XcorArgs& a, cudaStream_t st);

// Set the thread-local message returned by fc_last_error() (for entry points outside fc_api.cu).
// Network post-processing (k_post.cu): radix-select state in device scratch.
struct PostState {
    unsigned int max_key;  // largest magnitude (IEEE bits)
    unsigned int prefix;   // bits of the k-th largest magnitude found so far
    unsigned int mask;     // bits of prefix already fixed
    unsigned int pad_;
    long long k_rem;       // edges at the final magnitude still to keep
    long long k_total;     // edges to keep
    unsigned long long hist[256];
};
size_t post_scratch_bytes(long long P);
// Self-test: a bounded wait on an mbarrier nothing arrives at; sets ctrl->timeout.
cudaError_t launch_wait_probe(FcCtrl* ctrl, unsigned long long limit_ns, cudaStream_t st);
// Y[k] = M X[k] for count trials: M [n][C], X [count][C][N], Y [count][n][N].
cudaError_t launch_project(const float* M, const float* X, float* Y, int n, int C, int N, int count,
                           cudaStream_t st);
// Projection of band spectra: ring slot (pushed + write_from + t) % slots, [B][n], receives
// scale * M Xs[t] for t < count, Xs [count][B][C] (sensor spectra); scale = the session's
// prescale (1 before calibration).
cudaError_t launch_project_spectra(const float* M, const float2* Xs, float2* ring, int n, int C, int B, int count,
                                   int write_from, int slots, const FcCtrl* ctrl, cudaStream_t st);
// Kept normalized weights out[P], keep flags, degree[n] and strength[n] (both optional);
// synchronizes the stream.
cudaError_t launch_network_top(const float* w, long long P, int n, long long k, void* scratch, float* out,
                               int* degree, float* strength, int num_sms, cudaStream_t stream);

void fc_internal_set_error(const char* msg);
// Multiprocessor count of a device (device < 0: the current one), queried once per device
// and cached; 152 (GB300) only if the query fails.
int fc_device_sms(int device = -1);

// Streaming pushes of several sessions split into stages, for the serving engine
// (fc_server.cu): each trial is already on the device (x[i]). pre: validation, spectrum and
// per-node sums of all sessions, one launch per stage; the pair update is batched across
// sessions (launch_stream_batch with fc_push_stream_args); post: band reduction (if any),
// the drift re-sum slice, then one commit of all sessions with bookkeeping. Every session
// runs on the stream st; snap[i] (device-visible host memory, or NULL) receives session
// i's control block after its commit. Sessions that are uncalibrated, hold COR/XCOR or are
// in full mode take fc_push_single instead.
bool fc_push_needs_single(fc_session* s);
fc_status fc_push_single(fc_session* s, const float* xdev);
PairArgs fc_push_stream_args(fc_session* s);
fc_status fc_push_batch_pre(fc_session* const* ss, const float* const* x, int count, cudaStream_t st);
fc_status fc_push_batch_post(fc_session* const* ss, FcCtrl* const* snap, int count, cudaStream_t st);
// Launch, on each session's side stream, the drift re-sum slices that fc_push_batch_pre set
// up (call after the batched update launch, so the update's CTAs are dispatched first).
fc_status fc_push_batch_fork(fc_session* const* ss, int count);
void fc_count_launch(fc_session* s);
size_t fc_plan_session_bytes(int n, int N, int B, int W, uint32_t mask, fc_mode mode,
                             fc_precision prec = FC_PREC_FP32, int nfft = 0);
// Whether a session with these sizes computes its spectra by real FFT (method as configured;
// FC_SPECTRUM_AUTO: the cheaper one); 0 for an FFT request the sizes do not allow.
bool fc_spectrum_uses_fft(int N, int B, int nfft, fc_spectrum method);
bool fc_fft_size_ok(int nfft);
// Radices (4 first, then 2, 3, 5, 7) of m = nfft/2, four bits each; returns the pass count,
// or -1 when m has a prime factor above 7.
int fc_fft_radices(int m, unsigned long long* packed);
int fc_band_bins(double fs, fc_band band, int* first);

cudaError_t launch_expand_dense(const float* packed, float* dense, int n, int antisym,
                                cudaStream_t st);
cudaError_t launch_acc_field(const float* acc, const unsigned short* ta, const unsigned short* tb,
                             int ntp, int B, int n, int field, double* out, cudaStream_t st);
cudaError_t launch_df_planes_to_double(const float* acc2, long long P, double* out, cudaStream_t st);
