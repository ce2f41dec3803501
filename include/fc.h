/*
 * fc.h - C ABI of the GB300 (sm_103a) online all-to-all functional connectivity library.
 *
 * The library follows the statement of the problem in Esch et al., "Online functional
 * connectivity analysis of large all-to-all networks" (arXiv 2303.03279):
 *   - trials arrive as node x sample matrices (Methods 2.4, 2.5; Results 3.2.3: 265 x 250);
 *   - per trial, a spectrum per node, then the cross-spectral density CSD_xy = x y* and the
 *     power spectral density PSD_x = A_x^2 (Supplementary Information 1, Frequency Domain);
 *   - running sums of those over the trials being averaged (Methods 2.4: "the sums of CSD
 *     and PSD over all trials are directly computed"), only one half of the edge weights
 *     (Methods 2.4: undirected metrics);
 *   - the user sets the number of trials to average, and each new trial is added to the
 *     network (Methods 2.5; Results 3.2.3), with stored per-trial intermediates reused
 *     (Methods 2.4 storage mode; Discussion);
 *   - metrics COR, XCOR, COH, IMAGCOHY, PLV, PLI, USPLI, WPLI, DSWPLI (Methods 2.1,
 *     Supplementary Information 1), band-averaged over the selected frequency bins
 *     (Results 3.2.1, 3.2.3), returned as a network of nodes and weighted edges.
 *
 * Conventions (all entry points):
 *   - Every call returns an fc_status and never throws or aborts. On failure,
 *     fc_last_error() returns a thread-local, library-owned message.
 *   - The library owns only the session handle and the device memory it allocates for
 *     the session. Every input and output buffer belongs to the caller; the library
 *     copies inputs and never keeps a caller pointer past the call.
 *   - Work is enqueued on the session's CUDA stream (fc_config.stream, or a stream the
 *     library creates). Calls returning data into host memory synchronize that stream;
 *     calls with device outputs do not.
 *   - Pointers marked "host or device" are interpreted according to the *_on_device flag.
 *   - Node pairs are (i, j) with i < j. "Packed upper" layout: pair (i, j) at index
 *     p = i*n - i*(i+1)/2 + (j - i - 1), P = n*(n-1)/2 entries.
 *   - There is no CPU fallback: a session can only be created when a CUDA device is
 *     present; otherwise fc_session_create returns FC_ERR_CUDA.
 */
#ifndef FC_H
#define FC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fc_session fc_session; /* opaque, library-owned */

typedef enum {
    FC_OK = 0,
    FC_ERR_INVALID_ARG = -1,   /* a null pointer, a size out of range, a bad flag */
    FC_ERR_OUT_OF_MEMORY = -2, /* device or host allocation failed; nothing was changed */
    FC_ERR_CUDA = -3,          /* a CUDA runtime error (message in fc_last_error) */
    FC_ERR_NOT_READY = -4,     /* no trial has been accepted yet */
    FC_ERR_TIMEOUT = -5,       /* a bounded device-side wait ran out */
    FC_ERR_ADMISSION = -6,     /* a server refused a session: HBM budget exhausted */
    FC_ERR_NONFINITE = -7,     /* a pushed trial held NaN/Inf and was rejected */
    FC_ERR_UNSUPPORTED = -8    /* a valid request this build does not implement */
} fc_status;

/* Metric bits (Methods 2.1 list; definitions in Supplementary Information 1). */
enum {
    FC_COR = 1u << 0,      /* Pearson correlation, mean over trials */
    FC_XCOR = 1u << 1,     /* maximum normalised cross-correlation, mean over trials */
    FC_COH = 1u << 2,      /* |COHY| */
    FC_IMAGCOHY = 1u << 3, /* Im(COHY), antisymmetric: (j,i) = -(i,j) */
    FC_PLV = 1u << 4,      /* |mean of e^{i(Phi_x - Phi_y)}| */
    FC_PLI = 1u << 5,      /* |mean of sign(Im CSD)| */
    FC_USPLI = 1u << 6,    /* (K PLI^2 - 1)/(K - 1); NaN for K < 2 */
    FC_WPLI = 1u << 7,     /* |mean Im CSD| / mean |Im CSD| */
    FC_DSWPLI = 1u << 8    /* ((sum Im)^2 - sum Im^2)/((sum |Im|)^2 - sum Im^2) */
};
#define FC_SPECTRAL_METRICS (FC_COH | FC_IMAGCOHY | FC_PLV | FC_PLI | FC_USPLI | FC_WPLI | FC_DSWPLI)
#define FC_ALL_METRICS (FC_COR | FC_XCOR | FC_SPECTRAL_METRICS)

typedef enum {
    FC_TAPER_NONE = 0,
    FC_TAPER_HANN = 1,    /* periodic Hann, w(t) = 0.5 - 0.5 cos(2 pi t / N) */
    FC_TAPER_HANN_SYM = 2 /* symmetric Hann, w(t) = 0.5 - 0.5 cos(2 pi t / (N - 1)) */
} fc_taper;

/* Frequency band: every bin k (0 <= k <= nfft/2) with f_lo <= k*fs/nfft < f_hi.
 * nfft >= n_samples (the trial is zero-padded to nfft). */
typedef struct {
    double f_lo;
    double f_hi;
    int nfft;
} fc_band;

typedef enum {
    FC_PREC_FP32 = 0, /* every sum from exactly rounded FP32 terms, FP64-class accumulation */
    FC_PREC_TF32 = 1, /* linear sums (CSD, phasors) on tensor cores, TF32 operands, FP32 accumulate:
                         FC_MODE_FULL recomputes them each push; FC_MODE_STREAM (sliding window,
                         resum_period >= 0) keeps the exact streaming update and takes them from the
                         tensor cores in its drift re-sum (COH and PLV then carry the operand
                         rounding; IMAGCOHY, PLI, USPLI, WPLI, DSWPLI stay exact-term sums) */
    FC_PREC_BF16 = 2, /* same with BF16 operands */
    FC_PREC_FP16 = 3, /* same with FP16 operands */
    FC_PREC_TF32X3 = 4 /* split TF32: each operand a TF32 high part plus a TF32 low part, three
                          products per step (hi hi + hi lo + lo hi), FP32-class products; in
                          FC_MODE_FULL the linear metrics then match FP32 sessions to about
                          1e-6, in FC_MODE_STREAM COH and PLV keep that accuracy after a
                          re-sum instead of the single-operand rounding */
} fc_precision;

typedef enum {
    FC_MODE_STREAM = 0, /* resident accumulators; each push adds the new trial and
                           subtracts the one leaving the window (Methods 2.4 storage mode) */
    FC_MODE_FULL = 1    /* no accumulators; each push recomputes the window from the stored
                           spectra (the storage-off comparison of Results 3.1) */
} fc_mode;

/* How the band spectrum of a trial is computed (Methods 2.4: the per-trial spectrum of each
 * node); both give the same bins to FP32 rounding. */
typedef enum {
    FC_SPECTRUM_AUTO = 0, /* the cheaper of the two for the session's sizes */
    FC_SPECTRUM_DFT = 1,  /* band DFT: the trial times an [n_samples x n_bins] factor table
                             (taper folded in, angles reduced exactly in FP64 on the host); any nfft */
    FC_SPECTRUM_FFT = 2   /* real FFT of the tapered trial zero-padded to nfft (a mixed-radix
                             complex FFT of nfft/2 points and the even/odd split), then the band
                             bins selected; nfft even, 16 <= nfft <= 16384, nfft/2 with no prime
                             factor above 7 (e.g. 512, 600, 1000, 1024, 4200) */
} fc_spectrum;

typedef struct {
    fc_precision precision;
    fc_mode mode;
    void* stream;     /* cudaStream_t to enqueue on; NULL: the library creates one */
    int resum_period; /* stream mode: every accumulator is re-summed from the stored spectra
                         once per resum_period pushes (drift reset), spread as one slice of
                         1/resum_period of the tile pairs per push; 0 = the window length;
                         -1 = never */
    /* Optional device allocator (e.g. a framework's caching allocator). Both NULL: cudaMalloc. */
    void* (*dev_alloc)(size_t bytes, void* ctx);
    void (*dev_free)(void* ptr, void* ctx);
    void* alloc_ctx;
    fc_spectrum spectrum; /* FC_SPECTRUM_AUTO by default */
} fc_config;

typedef struct {
    int n_nodes, n_samples, n_bins, first_bin, nfft;
    int window;           /* W (0 = cumulative) */
    int k_used;           /* trials in the current window (after completed work) */
    long long pushes;     /* accepted pushes */
    long long rejected;   /* pushes rejected as non-finite */
    long long pairs;      /* P = n (n - 1) / 2 */
    size_t device_bytes;  /* device memory held by the session */
    uint32_t metric_mask;
    fc_mode mode;
    fc_precision precision;
    fc_spectrum spectrum; /* the method in use (FC_SPECTRUM_DFT or FC_SPECTRUM_FFT) */
} fc_info;

/* Fill *cfg with the defaults: FP32, stream mode, library stream, resum_period 0, cudaMalloc,
 * spectrum method chosen by the library. */
fc_status fc_config_default(fc_config* cfg);

/* Create a session (Methods 2.4/2.5 settings: nodes, samples, sampling rate, band, taper,
 * metrics, number of trials to average).
 *   n_nodes >= 2, 1 <= n_samples <= band.nfft, fs > 0, the band selects >= 1 bin;
 *   metric_mask: nonzero subset of FC_ALL_METRICS; the state of a family is allocated
 *     only when the mask holds one of its metrics (spectral: spectra ring and pair sums;
 *     COR: normalized-trial ring and its split-TF32 operand ring; XCOR: spectra ring and
 *     per-trial values), and only those metrics are computed per push; XCOR needs
 *     n_samples <= 8192 (its transforms run in registers up to 8192 complex points);
 *   window: W >= 0 trials (0 = cumulative; FC_MODE_FULL needs W >= 1);
 *   cfg: NULL for defaults. *out receives the handle; on failure *out is NULL and nothing
 *   stays allocated. Errors: FC_ERR_INVALID_ARG, FC_ERR_UNSUPPORTED (XCOR above 8192
 *   samples; FC_SPECTRUM_FFT with an nfft it does not take, see fc_spectrum),
 *   FC_ERR_OUT_OF_MEMORY, FC_ERR_CUDA. */
fc_status fc_session_create(int n_nodes, int n_samples, double fs, fc_band band, fc_taper taper,
                            uint32_t metric_mask, int window, const fc_config* cfg,
                            fc_session** out);

/* Synchronize the session's stream and free everything it holds. NULL is accepted. */
fc_status fc_session_destroy(fc_session* s);

/* Push one trial x[n_nodes][n_samples] (float32, row-major, host or device). The trial is
 * copied; a pageable host buffer may be reused on return, a page-locked one or a device
 * buffer once the session's stream has passed this call (fc_sync). A trial holding NaN or
 * Inf is rejected on the device and leaves the state unchanged; the next synchronizing
 * call (fc_sync, fc_get_network, fc_session_info) then reports FC_ERR_NONFINITE once.
 * In stream mode with a drift re-sum, the push's re-sum slice runs on a second stream the
 * session owns (created on first use, lowest priority), beside the update on the session's
 * stream; events order it after the push's spectra and before the push's end on the
 * session's stream, so callers see one ordered stream as before. */
fc_status fc_push_trial(fc_session* s, const float* x, int x_on_device);

/* Push `count` trials x[count][n_nodes][n_samples] (host or device) and update the network
 * once at the end. Same copying and rejection rules as fc_push_trial, per trial. */
fc_status fc_push_trials(fc_session* s, const float* x, int count, int x_on_device);

/* Band-averaged network of one metric (a single bit of the session's mask).
 *   packed_upper = 1: out[P] in the packed upper layout; 0: out[n][n] dense, diagonal 0,
 *   symmetric except IMAGCOHY (antisymmetric). out_len: element capacity of out.
 *   k_used (nullable) receives the number of trials the network averages.
 * Errors: FC_ERR_NOT_READY before the first accepted trial, FC_ERR_INVALID_ARG. */
fc_status fc_get_network(fc_session* s, uint32_t metric, int packed_upper, float* out,
                         size_t out_len, int out_on_device, int* k_used);

/* Start reading one metric's packed band-averaged network out[P] (the values after every
 * push enqueued so far) into host memory and return without waiting. The plane is first
 * copied on the device (4 P bytes at device bandwidth, on the session's stream), then moved
 * to `out` on a separate copy stream, so the transfer overlaps the pushes that follow.
 * Single host trials pushed with fc_push_trial are likewise copied in on their own stream
 * into alternating device buffers, so a loop of push, read-async, wait-for-the-previous
 * keeps the compute stream busy. `out` must stay valid until fc_network_wait returns for
 * it and should be page-locked (pinned) for the copy to overlap. At most two reads are in
 * flight: starting a third first waits for the oldest. Rejected trials are reported by the
 * synchronizing calls (fc_sync, fc_get_network), not here.
 * Errors: FC_ERR_NOT_READY before the first push, FC_ERR_INVALID_ARG, FC_ERR_CUDA. */
fc_status fc_get_network_async(fc_session* s, uint32_t metric, float* out, size_t out_len);

/* Wait until the oldest read started by fc_get_network_async has landed in host memory
 * (FC_OK at once when none is in flight). */
fc_status fc_network_wait(fc_session* s);

/* Per-bin values of one spectral metric, out[n_bins][P] (packed upper per bin). */
/* Post-processing of the current band-averaged network of one metric, as the paper
 * presents its networks (Results 3.1.2, 3.2.2: normalized by the maximum edge weight;
 * Results 3.2.2, 3.2.3: only the strongest 5 / 10 / 25 % of the edges; Introduction: node
 * degree and node strength). Edges are ranked by magnitude |w| (IMAGCOHY is signed);
 * kept = ceil(percent * P / 100) edges, among equal magnitudes the lower packed index
 * first; NaN edges count as 0.
 *   weights  [P] packed upper: w / max|w| for kept edges, 0 elsewhere (NULL: not returned)
 *   degree   [n] kept edges at each node; strength [n] sum of their normalized |w|
 *            (both NULL, or both given)
 * Outputs are host or device memory (out_on_device) and belong to the caller; the call
 * synchronizes the session's stream. Uses session-owned device scratch (allocated on
 * first use, about 5 B per pair). Errors: FC_ERR_INVALID_ARG (metric, percent, outputs),
 * FC_ERR_NOT_READY (nothing accepted yet), FC_ERR_NONFINITE (a rejection to report first). */
typedef struct {
    float max_abs;    /* the normalizer, max |w| over the edges (0: an all-zero network) */
    float threshold;  /* |w| of the weakest kept edge, before normalization (0 if none kept) */
    long long kept;   /* edges kept */
} fc_top_info;
fc_status fc_get_network_top(fc_session* s, uint32_t metric, double percent, float* weights,
                             int* degree, float* strength, int out_on_device, fc_top_info* info);

/* Change the band the networks average over to [f_lo, f_hi) Hz, a sub-band of the bins the
 * session computes (its creation band at the same nfft). The networks are refinalized from
 * the per-bin sums at once and every later push averages over the new band; no trial is
 * reprocessed in streaming mode (the per-bin accumulators hold everything; the Discussion,
 * section 4, contrasts this CSD/PSD design with methods that filter the signal to one band
 * before a Hilbert transform); full mode recomputes the window from its stored spectra. FC_ERR_INVALID_ARG if the band selects no bin or reaches
 * outside the computed ones (create the session with the wider band). */
fc_status fc_set_band(fc_session* s, double f_lo, double f_hi);

/* Session snapshot: the whole device state of a session (spectra ring, per-bin sums,
 * networks, control block, COR/XCOR state) and its window position, as one byte image in
 * caller-owned host memory, e.g. to checkpoint a long online session. fc_session_snapshot
 * synchronizes the session; fc_session_restore overwrites the state of a session created
 * with identical settings (FC_ERR_INVALID_ARG otherwise, or for a short or foreign buffer),
 * which then continues exactly as the snapshotted one would. The image is a header, the
 * buffer sizes and the buffers, in this library version's layout. */
fc_status fc_session_snapshot_size(fc_session* s, size_t* bytes);
fc_status fc_session_snapshot(fc_session* s, void* host_buf, size_t len);
fc_status fc_session_restore(fc_session* s, const void* host_buf, size_t len);

/* Source projection ahead of the spectrum (Methods 2.5, Figure 1: in the source-level
 * pipeline each trial is mapped to the source space by the inverse operator before the
 * connectivity step). op is M [n_nodes][n_channels], row-major, FP32, host or device
 * memory (copied). After this call every push takes sensor trials x[n_channels][n_samples]
 * (same host/device rules as before) and the session's nodes are the n_nodes sources:
 * y = M x per trial, FP32 on the CUDA cores, then validation, spectrum, COR/XCOR as usual.
 * op == NULL removes the projection (pushes take [n_nodes][n_samples] again). The operator
 * is configuration, not state: snapshots do not carry it. FC_ERR_INVALID_ARG for
 * n_channels < 1 with a non-NULL op. */
fc_status fc_set_projection(fc_session* s, const float* op, int n_channels, int op_on_device);

fc_status fc_get_network_bins(fc_session* s, uint32_t metric, float* out, size_t out_len,
                              int out_on_device);

/* Argmax lags of XCOR for the most recent trial, out[P] (int32, packed upper): for pair
 * (i, j) the lag tau of max_tau sum_t x_i(t + tau) x_j(t). Needs FC_XCOR in the mask. */
fc_status fc_get_xcor_lags(fc_session* s, int32_t* out, size_t out_len, int out_on_device);

/* Switch the set of finalized metrics (Results 3.2.3: metrics switched on the fly). The
 * accumulators are shared, so a switch recomputes only the networks. Time-domain bits
 * (COR, XCOR) can only be kept or removed, not added after creation; spectral bits cannot
 * be added to a session created without any (it holds no spectra or pair sums). */
fc_status fc_set_metric_mask(fc_session* s, uint32_t metric_mask);

/* Wait for the session's stream; reports a pending FC_ERR_NONFINITE. */
fc_status fc_sync(fc_session* s);

/* Session facts (synchronizes). */
fc_status fc_session_info(fc_session* s, fc_info* info);

/* Thread-local message of the last failing call on this thread ("" if none). */
const char* fc_last_error(void);

/* ---- measurement hooks ------------------------------------------------------------ */

/* Kernel ids reported by fc_kernel_times. */
typedef enum {
    FC_K_SPECTRUM = 0, /* taper + band DFT of one or more trials */
    FC_K_CALIBRATE,    /* one-time power-of-two prescale of the spectra */
    FC_K_NODE,         /* per-node PSD sums */
    FC_K_STREAM,       /* streaming add/subtract update with fused finalize */
    FC_K_WINDOW,       /* CUDA-core full-window sums (all terms) with fused finalize */
    FC_K_HERK_TC,      /* tensor-core Hermitian rank-K linear sums */
    FC_K_BAND_REDUCE,  /* band average of per-bin-group partial sums */
    FC_K_COR,          /* correlation products */
    FC_K_XCOR,         /* cross-correlation via FFT */
    FC_K_PROJECT,      /* source projection of sensor trials */
    FC_K_OTHER,
    FC_K_COUNT
} fc_kernel_id;

typedef struct {
    int launches;
    double total_ms;
} fc_kernel_time;

/* Enable (1) or disable (0) per-launch CUDA-event timing on the session's stream. */
fc_status fc_set_profiling(fc_session* s, int enable);

/* Accumulated per-kernel timings since profiling was enabled or reset (synchronizes).
 * out[FC_K_COUNT]. reset = 1 clears the counters after reading. */
fc_status fc_kernel_times(fc_session* s, fc_kernel_time* out, int reset);

/* Total kernel launches this session has enqueued. */
long long fc_launch_count(const fc_session* s);

/* The session's CUDA stream (cudaStream_t), e.g. to record events on it. */
void* fc_session_stream(const fc_session* s);

/* ---- test hooks ------------------------------------------------------------------- */

/* Spectra of the trial pushed `age` accepted pushes ago (0 = newest), as the kernels hold
 * them (after the session's power-of-two prescale): out[n_bins][n_nodes][2] (re, im). */
fc_status fc_debug_get_spectra(fc_session* s, int age, float* out, size_t out_len);

/* The power-of-two factor the spectra were multiplied by (all metrics are invariant). */
fc_status fc_debug_get_scale(fc_session* s, float* scale);

/* Accumulator fields (stream mode), each out[n_bins][P] in double (hi + lo of the
 * double-float pairs); FC_ACC_PSD gives out[n_bins][n_nodes]. */
typedef enum {
    FC_ACC_CSD_RE = 0, FC_ACC_CSD_IM, FC_ACC_U_RE, FC_ACC_U_IM, FC_ACC_ABS, FC_ACC_SQ,
    FC_ACC_SIGN, FC_ACC_PSD, FC_ACC_COR, FC_ACC_XCOR
} fc_acc_field;
/* Self-test of failure detection: a kernel waits, through the library's bounded-wait
 * routine, on a device barrier that nothing completes, with a budget of limit_ms (0 < limit
 * <= 1000). The wait gives up, the kernel records a timeout in the session's control block
 * and returns (no fault, the context stays usable); the call then returns FC_ERR_TIMEOUT,
 * as any call would after a real wait ran out. The session reports FC_ERR_TIMEOUT from then
 * on: use a throwaway session. */
fc_status fc_debug_wait_probe(fc_session* s, double limit_ms);

fc_status fc_debug_get_accumulators(fc_session* s, fc_acc_field field, double* out,
                                    size_t out_len);

/* ---- serving: many concurrent sessions, continuous batching ----------------------- */
/*
 * A server holds many sessions resident on one GPU and turns every arriving trial of any
 * session into a request (the paper's online setting, Methods 2.5 / Results 3.2.3: each
 * new trial is added to the network as it arrives, under a per-block deadline). A worker
 * thread runs ticks; each tick is one launch of the persistent streaming kernel over a
 * share of the pushes of up to max_batch sessions (FIFO within a session, one trial in
 * progress per session). A launch carries at most launch_blocks state blocks; a larger push
 * is split over consecutive launches and its trial completes with the last one, so the
 * trials of small sessions are not held back by a large session's push. Trials arriving
 * while a launch runs join the next one, and up to two launches are in flight, so host
 * staging overlaps the device work. Sessions are admitted against a device-memory budget.
 * Results are identical whichever sessions share a launch.
 */
typedef struct fc_server fc_server;

typedef struct {
    size_t hbm_budget; /* device bytes the server may hold for sessions (0: no limit) */
    int max_batch;     /* sessions per launch, 1..32 (0: 32) */
    int plain;         /* 1: comparison mode - FC_MODE_FULL FP32 sessions, one trial at a time,
                          each a full-window recompute (no batching, no streaming sums) */
    int launch_blocks; /* state blocks (one 32 x 32 tile pair x one bin, 106 KB of traffic)
                          per launch: 0 = 65536 (about 1.2 ms on GB300); < 0 = no limit */
    fc_precision precision; /* streaming sessions (plain = 0): FC_PREC_FP32 (default), or a
                          tensor-core precision whose drift re-sum takes the linear sums from
                          the tensor cores (see fc_config.precision) */
} fc_server_config;

typedef struct {
    int session;       /* server session id */
    long long seq;     /* index of the trial within its session's submissions (0-based) */
    fc_status status;  /* FC_OK; FC_ERR_NONFINITE: the trial held NaN/Inf and was rejected
                          (the session state is unchanged); FC_ERR_TIMEOUT: a bounded device
                          wait ran out */
    double arrival_ms; /* the submitter's arrival stamp */
    double done_ms;    /* when the server observed the network ready (same clock) */
    int batch;         /* sessions in the streaming-kernel launch that completed this trial
                          (1: it ran alone, e.g. a session's first, calibrating push) */
} fc_result;

typedef struct {
    long long submitted, completed;
    long long launches;         /* ticks with device work */
    long long batched_trials;   /* session shares over all ticks */
    long long pair_bin_updates; /* sum of P * B over trials completed with FC_OK */
    size_t hbm_used;
    int sessions;
} fc_server_stats;

/* Milliseconds on the server's clock (steady, process-wide); use it for arrival stamps. */
double fc_server_now_ms(void);

fc_status fc_server_create(const fc_server_config* cfg, fc_server** out);

/* Open a session (same settings as fc_session_create, streaming mode, the server's precision). Returns
 * FC_ERR_ADMISSION without allocating when its device memory would exceed the budget;
 * the caller may retry after closing sessions. *session_id receives the id. */
fc_status fc_server_open(fc_server* sv, int n_nodes, int n_samples, double fs, fc_band band,
                         fc_taper taper, uint32_t metric_mask, int window, int* session_id);

/* Device bytes a session with these settings would hold (the admission figure). */
fc_status fc_server_session_bytes(int n_nodes, int n_samples, double fs, fc_band band,
                                  uint32_t metric_mask, int window, int plain, size_t* bytes);

/* Queue one trial x[n_nodes][n_samples] (host memory, copied before return). */
fc_status fc_server_submit(fc_server* sv, int session_id, const float* x, double arrival_ms);

/* Completed trials, oldest first: up to max results into out; waits up to wait_ms for at
 * least one (0: no wait). */
fc_status fc_server_poll(fc_server* sv, fc_result* out, int max, int* n_out, int wait_ms);

/* Wait until every submitted trial has completed (up to timeout_ms; FC_ERR_TIMEOUT after). */
fc_status fc_server_drain(fc_server* sv, int timeout_ms);

/* Current band-averaged network of a session (packed upper, host memory), after its last
 * trial whose push is fully enqueued; waits while a push is split between launches. */
fc_status fc_server_get_network(fc_server* sv, int session_id, uint32_t metric, float* out,
                                size_t out_len);

/* Finish the session's queued trials and free its memory (returns it to the budget). */
fc_status fc_server_close(fc_server* sv, int session_id);

fc_status fc_server_stats_get(fc_server* sv, fc_server_stats* st);

/* Stop the worker, close every session, free everything. NULL is accepted. */
fc_status fc_server_destroy(fc_server* sv);

/* ---- FIR filtering of the incoming stream (upstream of the sessions) ------------- */
/*
 * Methods 2.4 (Noise Reduction plug-in): low-, high- and band-pass FIR filters designed on
 * the fly from the cut-offs, the transition bandwidth and the number of taps, all with a
 * linear phase, applied to the data blocks as they arrive with overlap-add across block
 * boundaries. Design: window method - the ideal response (differences of sinc low-passes)
 * times a Hamming window, odd length T (n_taps, rounded up to odd; 0: ceil(3.3 fs /
 * transition_hz)), at most 8191, computed in FP64 on the host and applied in FP32.
 * fc_fir_process filters one block x[n_channels][block_len] into y (host or device memory,
 * both on the same side): y[c][t] = sum_k h[k] x[c][t - k] over the continuous stream, the
 * state (the last T - 1 samples of every channel) carrying over between calls, so any
 * division into blocks gives the same output (a delay of (T - 1) / 2 samples). Host buffers
 * synchronize; device buffers are asynchronous on the given stream (NULL: the filter's own).
 */
typedef struct fc_fir fc_fir;
typedef enum { FC_FIR_LOWPASS = 0, FC_FIR_HIGHPASS = 1, FC_FIR_BANDPASS = 2 } fc_fir_kind;
/* lowpass uses f_hi, highpass f_lo, bandpass both; cut-offs inside (0, fs / 2). */
fc_status fc_fir_create(int n_channels, double fs, fc_fir_kind kind, double f_lo, double f_hi,
                        double transition_hz, int n_taps, void* stream, fc_fir** out);
/* The FP64 taps (T of them; taps may be NULL to ask for T only). */
fc_status fc_fir_get_taps(fc_fir* f, double* taps, int max_taps, int* n_taps);
fc_status fc_fir_process(fc_fir* f, const float* x, float* y, int block_len, int on_device);
/* Forget the stream so far (zero state). */
fc_status fc_fir_reset(fc_fir* f);
fc_status fc_fir_destroy(fc_fir* f);

/* ---- allocation-free entry point ------------------------------------------------ */

/* Size of the device scratch array behind fc_window_networks_noalloc (16 MiB). */
#define FC_NOALLOC_SCRATCH_BYTES (16u << 20)

/* Band-averaged spectral networks of one window, computed without allocating anything.
 * The paper has no counterpart to this call; it exists for callers that must not call
 * cudaMalloc: a real-time acquisition loop where an allocation (which can synchronize
 * the whole device and take an unbounded time) would miss the per-trial deadline, or a
 * host application whose device memory is owned by another allocator (a framework's
 * caching allocator, a pre-reserved pool).
 *
 *   spectra:  device pointer, [n_trials][n_bins][n_nodes] complex values stored as
 *             (re, im) float pairs - the layout of the library's own spectra (see
 *             fc_debug_get_spectra). The window is all n_trials trials.
 *   metric_mask: nonzero subset of FC_SPECTRAL_METRICS.
 *   out:      device pointer, out[7][P] (P = n_nodes (n_nodes - 1) / 2, packed upper
 *             per plane) in the order COH, IMAGCOHY, PLV, PLI, USPLI, WPLI, DSWPLI; only
 *             the planes of metrics in the mask are written. out_len: element capacity.
 *   stream:   cudaStream_t to enqueue on (NULL: the legacy default stream). The call is
 *             asynchronous; results are ready when the stream reaches this point.
 *
 * The spectra may be in any unit: as a session does with its own, the call scales them by
 * the power of two that brings their largest |re|, |im| into [1, 2) (exact; every metric
 * is invariant to it) as the kernels read them; the caller's buffer is not written. The
 * values must be finite: they are not checked, and a NaN or Inf gives NaN in the networks
 * of the pairs of its node (the call still returns FC_OK).
 *
 * Every intermediate (window control block, per-node PSD sums, tile tables, band
 * partial sums) lives in one file-scope device array of FC_NOALLOC_SCRATCH_BYTES that
 * every GPU loading the library holds until the process exits. Limits: the PSD sums and
 * tile tables must fit in it (n_bins * n_nodes below about 1.3 million); the band-partial
 * work split shrinks to what fits. Sizes beyond the limit return FC_ERR_INVALID_ARG with a
 * message in fc_last_error(). The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current; make that first call before
 * any stream capture (a failed lookup is not kept: the next call tries again). All calls
 * share the array and it keeps the last call's contents (the control block is cleared on
 * every call): calls whose work overlaps on the GPU (different streams, no ordering
 * between them) race and corrupt each other.
 * No cudaMalloc, cudaFree or allocating library routine is called. */
fc_status fc_window_networks_noalloc(const float* spectra, int n_trials, int n_bins, int n_nodes,
                                     uint32_t metric_mask, float* out, size_t out_len, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* FC_H */
