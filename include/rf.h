/*
 * rf.h -- C ABI of the ratio-filter library (librf.so), sm_103a.
 *
 * The library computes the data-parallel hot path of the ratio filter
 * (Murakami, Ghosh & Morisaki, "Efficient Reconstruction of Matched-Filter SNR
 * Time Series from Nearby Templates for CBC Searches"):
 *
 *   rf_mf_reference         complex SNR z_ref(t) of reference templates
 *                           (Sec. II.A, Eqs. 2-4 and 6)
 *   rf_build_ratio_kernels  truncated ratio kernels of the neighbours of one
 *                           reference (Sec. II.B-II.D, Eqs. 5, 7, 9, 10)
 *   rf_reconstruct          neighbour SNR series z = z_ref (*) r (Eq. 8)
 *   rf_reconstruct_winmax   the same, reduced on the fly to per-window
 *                           max|z|^2 and its first index (the peak read in Sec. IV)
 *
 * Conventions shared by every call
 * --------------------------------
 * Grid.  n samples (a power of two, 2^8..2^24) at fs Hz; dt = 1/fs, T = n dt,
 *   df = 1/T; one-sided bins f_k = k df, k = 0..n/2.  Fourier sign as in Eq. (1):
 *   forward transforms use exp(-2 pi i f t).
 * Data types.  grid.dtype selects the arithmetic of the whole path:
 *   RF_F64: real data double, complex data interleaved double2 (complex128);
 *   RF_F32: real data float,  complex data interleaved float2  (complex64).
 *   Template phases, their differences and all normalisation sums are FP64 in
 *   both modes.
 * Memory.  Unless stated otherwise a pointer argument is caller-owned DEVICE
 *   memory, 16-byte aligned, on the device that was current at rf_create.
 *   Host arrays are marked "host".  Opaque handles own their memory and are
 *   released with the matching free/destroy call.
 * Streams.  rf_stream is a cudaStream_t (NULL: the legacy default stream).
 *   Calls enqueue work on that stream and return without synchronising,
 *   except where a call says it synchronises.
 * Errors.  Every call returns an rf_status; on failure nothing has been
 *   enqueued and rf_last_error() (per host thread) describes why.  Arguments
 *   are validated on the host before any launch; no call aborts the process.
 *   RF_ECUDA reports a CUDA runtime error (message included).
 * Threads.  One rf_ctx must not be used by two host threads at once; different
 *   contexts may be used from different host threads concurrently (the library's
 *   process-wide state is counters, a driver entry point looked up once, and
 *   per-function launch attributes set to constant bounds).
 *   rf_mf_reference_noalloc is the exception: its static workspace is shared by
 *   every caller.
 * Sizes.  Device buffers are plain pointers: the caller provides at least the
 *   element counts each call states; the library cannot check a buffer's extent.
 */
#ifndef RF_H
#define RF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RF_ABI_VERSION 5

typedef struct rf_ctx rf_ctx;
typedef struct rf_kernels rf_kernels;
typedef void* rf_stream;

typedef enum {
  RF_OK = 0,
  RF_EINVAL = -1,        /* invalid argument (null, misaligned, out of range, wrong state) */
  RF_ENOMEM = -2,        /* device or host allocation failed */
  RF_ECUDA = -3,         /* CUDA runtime error */
  RF_ETIMEOUT = -4,      /* a bounded device-side wait ran out (status word) */
  RF_EUNSUPPORTED = -5   /* valid request this build does not implement */
} rf_status;

typedef enum { RF_F64 = 0, RF_F32 = 1 } rf_dtype;

/* Reconstruction algorithm.  AUTO picks per kernel-length bucket. */
typedef enum {
  RF_ALGO_AUTO = 0,
  RF_ALGO_DIRECT = 1,    /* direct time-domain sum on CUDA cores (Eq. 8) */
  RF_ALGO_OS = 2,        /* overlap-save block FFT (frequency form, Eq. 7), FP32 */
  RF_ALGO_GEMM = 3,      /* direct sum as a Hankel x taps complex GEMM on the tcgen05 tensor
                            cores (n a multiple of 128) */
  RF_ALGO_OS_BINS = 4    /* bucket form only (rf_kernels_prepare_forms): two-phase overlap-save,
                            the partition sums per bin over runs of output blocks, then the
                            block transforms; for kernels of many partitions */
} rf_algo;

/* Arithmetic of the reconstruction.  RF_PREC_NATIVE: the grid dtype on CUDA cores (direct,
 * overlap-save).  The tensor-core form (RF_ALGO_GEMM) splits every z_ref and tap value into
 * BF16 terms x = x0 + x1 + x2 (x_k = bf16 of the remainder) and accumulates in FP32:
 * RF_PREC_BF16 keeps x0 y0 (plain BF16, about 3 significant digits), RF_PREC_BF16X3 adds
 * x0 y1 + x1 y0, RF_PREC_BF16X6 adds x0 y2 + x1 y1 + x2 y0, RF_PREC_BF16X9 all nine products.
 * RF_PREC_3XTF32 splits into two TF32 terms (x0 = tf32(x), x1 = tf32(x - x0), round to
 * nearest) and keeps x0 y0 + x0 y1 + x1 y0 on the TF32 tensor pipe (half the BF16 rate). */
typedef enum {
  RF_PREC_NATIVE = 0,
  RF_PREC_BF16 = 1,
  RF_PREC_BF16X3 = 2,
  RF_PREC_BF16X6 = 3,
  RF_PREC_BF16X9 = 4,
  RF_PREC_3XTF32 = 5
} rf_prec;

/* A non-spinning stationary-phase inspiral (App. A, Eq. A1): h(f) = B(f) exp(-i Psi(f)),
 * B(f) = f^(-7/6) (unit scale: every SNR is normalised), Psi the TaylorF2 phase with
 * component masses m1, m2 in solar masses, coalescence time tc (s) and phase phic (rad). */
typedef struct {
  double m1, m2, tc, phic;
} rf_template;

/* The analysis grid and band.  f_high + df_high must not exceed fs/2.  The data band is
 * [f_low, f_high] (Eq. 4); the kernel window (Eq. 9) tapers over df_low below f_low and
 * df_high above f_high, with df_low = min(df_low_max, f_low/2, 1/sqrt|d tau'(f_low)|)
 * (Eq. 10).  pn_order: 0..7 (2 = 1PN, 7 = 3.5PN).  dtype: rf_dtype. */
typedef struct {
  int64_t n;
  double fs, f_low, f_high, df_high, df_low_max;
  int32_t pn_order;
  int32_t dtype;
} rf_grid;

/* ABI version (RF_ABI_VERSION) of the loaded library. */
int32_t rf_version(void);

/* Number of CUDA kernels this library has launched in this process (all threads). */
uint64_t rf_launch_count(void);

/* Message of the last failing call on this host thread ("" if none). Borrowed. */
const char* rf_last_error(void);

/* Create a context for one grid on the current device.  Allocates the FFT twiddle
 * tables and workspaces (about 40 n bytes).  Caller frees with rf_destroy. */
rf_status rf_create(const rf_grid* grid, rf_ctx** out);

/* Release a context and everything it owns.  Waits for the device.  NULL is a no-op. */
void rf_destroy(rf_ctx* ctx);

/* Largest workspace the context will use for `k_max` kernels (bytes), and reserve it now
 * (allocation happens here, never later in an rf_reconstruct* call of at most k_max kernels;
 * needed before capturing reconstruct calls in a CUDA graph).  Includes the tensor-core
 * form's Hankel core-matrix records of z_ref for its longest kernels (min(n, 65536) taps:
 * about 128 (n + min(n, 65536) + 1300) bytes, the 3xTF32 layout being the largest). */
rf_status rf_reserve(rf_ctx* ctx, int32_t k_max, int64_t* bytes_out);

/* Template spectrum h~(f_k) = B(f_k) exp(-i Psi(f_k)), k = 0..n/2, 0 at DC (App. A, Eq. A1).
 * h_out: complex[n/2+1] (grid dtype).  Phase in FP64.  Async on stream. */
rf_status rf_template_fd(rf_ctx* ctx, const rf_template* tmpl, void* h_out, rf_stream stream);

/* Reference matched filter (Sec. II.A, Eqs. 2-4, 6).  For each of the nref templates:
 *   N^2 = 4 df sum_{f_low<=f_k<=f_high} |h~_k|^2 inv_psd[k]             (Eq. 3, FP64)
 *   z[i] = (4 df / N) sum_{k=0}^{n/2} x~_k conj(h~_k) inv_psd[k] band_k exp(+2 pi i i k / n)
 * with x~_k = dt sum_j x[j] exp(-2 pi i j k / n) computed once for all references.
 * x: real[n] (grid dtype); inv_psd: double[n/2+1], 1/S_n(f_k) (values outside the band are
 * ignored: Eq. 4); refs: host array of nref templates; z_out: complex[nref][n] (grid dtype);
 * sigma_out: double[nref] (device, N of each reference).  Async on stream. */
rf_status rf_mf_reference(rf_ctx* ctx, const void* x, const double* inv_psd, int32_t nref,
                          const rf_template* refs, void* z_out, double* sigma_out, rf_stream stream);

/* Stored reference filters for rf_mf_filtered (the data-independent half of Eq. 2, kept like
 * the ratio kernels): per reference r and bin k = 0..n/2,
 *   filt[r][k] = (4 / (n N_r)) conj(h~_r(f_k)) inv_psd[k] on [f_low, f_high], 0 elsewhere,
 * with N_r as in rf_mf_reference (Eq. 3, FP64) and the phase in FP64, rounded once to the
 * grid dtype.  filt_out: complex[nref][n/2+1] (grid dtype); sigma_out: double[nref] (device,
 * may be NULL).  refs: host.  Async on stream. */
rf_status rf_reference_filters(rf_ctx* ctx, const double* inv_psd, int32_t nref, const rf_template* refs,
                               void* filt_out, double* sigma_out, rf_stream stream);

/* Reference matched filter from stored filters: X = DFT(x) once (unnormalised, Eq. 1), then
 * for each reference z_r[i] = sum_{k=0}^{n/2} X[k] filt[r][k] exp(+2 pi i i k / n), which is
 * z_ref of rf_mf_reference (Eqs. 2, 6).  The product is formed inside the first pass of the
 * inverse transform.  x: real[n]; filt: complex[nref][n/2+1]; z_out: complex[nref][n] (grid
 * dtype).  The first call allocates a temporary of up to min(nref, 2^27 / n) x n complex
 * values (later calls with as many references reuse it, so a warmed-up call can be captured
 * in a CUDA graph).  Async on stream. */
rf_status rf_mf_filtered(rf_ctx* ctx, const void* x, int32_t nref, const void* filt, void* z_out, rf_stream stream);

/* Ratio kernels of k neighbours of one reference (Sec. II.B-II.D).  Per neighbour j, in FP64:
 *   K~_k = (N_ref/N_j) W(f_k) conj(h~_j(f_k) / h~_ref(f_k))   (Eqs. 5, 7 and window Eq. 9)
 *   rho[m] = (1/n) sum_{k=0}^{n/2} K~_k exp(+2 pi i k m / n),  m = 0..n-1
 * then truncation, chosen by the flags `relative` (RF_TRUNC_RELATIVE | RF_TRUNC_ANALYTIC):
 * numeric (default): with a = max|rho|^2, the kept lags are those with |rho|^2 >= thr^2 a
 * (RF_TRUNC_RELATIVE) or |rho|^2 >= thr^2; the kernel is the shortest circular arc
 * [m0, m0+L) covering them (ties: smallest m0 in (-n/2, n/2]).
 * analytic (RF_TRUNC_ANALYTIC; Sec. II.D with the App. A expressions): a threshold amplitude
 * A on |r| = 2 fs |rho| / (N_ref/N_j) (1/s), A = thr max|r| with RF_TRUNC_RELATIVE, else
 * A = thr (the paper's threshold amplitude); for the four taper ends f_e = f_low - df_low,
 * f_low, f_high, f_high + df_high (taper widths df_e = df_low, df_low, df_high, df_high), with
 * c_e = -(Psi_j'(f_e) - Psi_ref'(f_e)) / (2 pi) and d_e = (R(f_e) / (4 pi df_e^2 A))^(1/3)
 * (R = B_j / B_ref), the kept lag times run from min(c_e - d_e) to max(c_e + d_e): lags
 * floor(min fs) .. ceil(max fs), m0 signed in (-n/2, n/2] (a span as long as the grid keeps the
 * whole grid from lag 0).  The
 * App. A bounds are asymptotic, so A should leave the reach well past the taper widths (the
 * paper's absolute 1e-3 / s, or a relative threshold of 1e-4 or less).
 * RF_KERNEL_REAL: the paper's real-kernel form (Eq. 8 with r(t) = 2 Re of the App. A integrand):
 * rho is replaced by 2 Re rho before truncation, which then acts on |2 Re rho| (analytic:
 * |r| = fs |2 Re rho| / (N_ref/N_j)).  z_ref has no negative-frequency content, so untruncated
 * the result equals the complex kernel's; truncated, the two differ.  The set then stores its
 * taps as REAL values of the grid dtype (half the bytes; rf_kernels_is_real reports it), the
 * direct form multiplies complex z_ref by real taps (half the multiply-adds), and the
 * overlap-save preparation keeps the Hermitian half of each partition spectrum (bins 0..B/2).
 * The tensor-core form builds its complex operands from the real taps (same cost).
 * Taps c[l] = rho[m0+l] are stored packed (grid dtype) with int32 signed m0 and length L per
 * neighbour.
 * Normalisation: the templates are the stationary-phase family A f^-7/6 e^{-i Psi} on one band,
 * so N_j / N_ref = A_j / A_ref and the factor (N_ref/N_j) |h~_j / h~_ref| is exactly 1 for any
 * amplitude scales: K~ = W e^{+i (Psi_j - Psi_ref)}, and inv_psd (validated like every
 * argument) does not change the taps.
 * Build grid (Sec. II.D: a kernel needs a frequency grid only as fine as its duration):
 * n_build = 0 builds on the data grid (n bins, the definition above); a power of two in
 * [16, n] builds every kernel on that grid (K~ at f_k = k fs / n_b, an n_b-point inverse
 * transform with the 1/n_b factor, lags signed in (-n_b/2, n_b/2]); -1 picks per neighbour the
 * smallest power of two of at least four times its lag extent (time offsets (Psi_j' -
 * Psi_ref')/(2 pi) at f_low - df_low and f_high + df_high, times fs, plus 4 fs / df_low),
 * capped at n.  RF_EINVAL for other n_build, for flags
 * outside RF_TRUNC_RELATIVE | RF_TRUNC_ANALYTIC | RF_KERNEL_REAL, and for an analytic threshold
 * of 0.
 * refs/nbrs: host; inv_psd: device double[n/2+1].  SYNCHRONISES `stream` (the lengths are
 * read back).  *out is freed with rf_kernels_free. */
#define RF_TRUNC_RELATIVE 1
#define RF_TRUNC_ANALYTIC 2
#define RF_KERNEL_REAL 4
rf_status rf_build_ratio_kernels(rf_ctx* ctx, const rf_template* ref, const rf_template* nbrs,
                                 int32_t k, const double* inv_psd, double threshold,
                                 int32_t relative, int64_t n_build, rf_kernels** out, rf_stream stream);

/* Import k kernels computed earlier and kept on disk or in host memory (Sec. II.B keeps the
 * truncated ratio waveforms between analyses):
 * lag0/len: host int32[k]; taps: HOST complex (grid dtype), packed back to back, sum(len)
 * entries.  Synchronous copy. */
rf_status rf_kernels_import(rf_ctx* ctx, int32_t k, const int32_t* lag0, const int32_t* len,
                            const void* taps, rf_kernels** out);

/* As rf_kernels_import for real-form kernels (RF_KERNEL_REAL): taps are HOST real values of
 * the grid dtype (double or float), sum(len) of them. */
rf_status rf_kernels_import_real(rf_ctx* ctx, int32_t k, const int32_t* lag0, const int32_t* len,
                                 const void* taps, rf_kernels** out);

/* *real = 1 when the set holds real-form taps (built with RF_KERNEL_REAL or imported with
 * rf_kernels_import_real), else 0.  RF_EINVAL if either pointer is NULL. */
rf_status rf_kernels_is_real(const rf_kernels* kern, int32_t* real);

/* Borrowed views of a kernel set: host arrays len[k], lag0[k], offset[k+1] (int64) and
 * df_low[k] (Hz; NaN for imported kernels), and the device tap buffer (grid dtype complex, or
 * grid dtype real for a real-form set).
 * Any output pointer may be NULL. */
rf_status rf_kernels_info(const rf_kernels* kern, int32_t* k, const int32_t** len,
                          const int32_t** lag0, const int64_t** offset, const double** df_low,
                          const void** taps_dev);

/* Prepare a kernel set for overlap-save reconstruction (Eq. 7 in blocks; RF_F32 grids,
 * n >= 512): block size B (a power of two in [512, 32768], <= n) and partition length Lp
 * (B/2, B/4 or B/8 taps; B/2 or B/4 at 32768, whose blocks run on pairs of CTAs of a thread
 * block cluster, each transforming the bins of one parity); 0 for either picks, among the allowed layouts, the one of least
 * modelled cost for this set's kernel lengths (a per-block cost table measured on GB300,
 * plus a penalty for launches too small to fill the GPU).  Computes the partition spectra
 * FFT_B(taps)/B in FP64 and stores them as complex64 inside the kernel set
 * (sum_j ceil(L_j / Lp) x B complex64; for a real-form set the Hermitian half, bins 0..B/2 in
 * rows of B/2 + 8, and block sizes up to 16384).  Each output block transform then keeps B - Lp
 * outputs.  The first overlap-save reconstruction prepares with the modelled choice if this
 * was not called.  Allocates; SYNCHRONISES `stream`.  RF_EINVAL for other sizes. */
rf_status rf_kernels_prepare(rf_ctx* ctx, rf_kernels* kern, int32_t block, int32_t part, rf_stream stream);

/* Overlap-save layout a kernel set is prepared for: block size and partition length of its
 * first length bucket (both 0 when not prepared).  Either output pointer may be NULL. */
rf_status rf_kernels_os_layout(const rf_kernels* kern, int32_t* block, int32_t* part);

/* Overlap-save preparation with a layout per kernel-length bucket: bucket b takes the
 * neighbours with cuts[b] <= L < cuts[b+1] (cuts[0] = 0, increasing; the last bucket is open)
 * and runs with block size blocks[b] and partition length parts[b] (each as in
 * rf_kernels_prepare, both non-zero).  A reconstruction then makes one segment transform and
 * one launch per bucket; rows keep the neighbour order.  1 <= nb <= 8; cuts, blocks, parts are
 * host arrays.  Allocates; SYNCHRONISES `stream`. */
rf_status rf_kernels_prepare_buckets(rf_ctx* ctx, rf_kernels* kern, int32_t nb, const int32_t* cuts,
                                     const int32_t* blocks, const int32_t* parts, rf_stream stream);

/* Preparation with a form per kernel-length bucket (bucket b: cuts[b] <= L < cuts[b+1], cuts as in
 * rf_kernels_prepare_buckets): algos[b] = RF_ALGO_OS runs overlap-save with block size blocks[b]
 * and partition length parts[b]; RF_ALGO_GEMM runs the tensor-core form at the split precision
 * precs[b] with the tile layout (blocks[b] neighbours per group, parts[b] output tiles stacked
 * per MMA): (16, widest stack) or (widest group, 1), or (0, 0) for the library's rule; kernels of
 * at most 65536 taps; RF_ALGO_OS_BINS runs two-phase overlap-save (the partition sums per bin,
 * then the block transforms; blocks[b] of 4096, 8192 or 16384 with parts[b] = blocks[b]/2 or /4,
 * or 32768 with 16384; its waves run phase 2 on a stream of the context's own, joined back to
 * `stream` by events, so a captured call still forms one graph); RF_ALGO_DIRECT runs the
 * CUDA-core direct sum.  The overlap-save buckets
 * share one segment transform per layout and launch as rf_kernels_prepare_buckets; each other
 * bucket runs on a kernel set holding just its neighbours (taps copied, tensor-core operands
 * prepared here) into a temporary whose rows are then scattered to the neighbours' rows, so a
 * reconstruction of the set (RF_ALGO_AUTO or RF_ALGO_OS; rf_reconstruct, _winmax, _batched) mixes
 * forms within one call.  The temporary (rows x windows, or rows x n for the series form) is
 * sized on the first call: make one before capturing a CUDA graph.  RF_F32 grids, n >= 512.
 * Allocates; SYNCHRONISES `stream`.  RF_EINVAL for invalid forms, layouts or lengths. */
rf_status rf_kernels_prepare_forms(rf_ctx* ctx, rf_kernels* kern, int32_t nb, const int32_t* cuts,
                                   const int32_t* algos, const int32_t* precs, const int32_t* blocks,
                                   const int32_t* parts, rf_stream stream);

/* The form (rf_algo) and precision of each bucket of a prepared kernel set, up to max_nb, and
 * their number into *nb (0 when not prepared); any output pointer may be NULL. */
rf_status rf_kernels_bucket_forms(const rf_kernels* kern, int32_t max_nb, int32_t* algos, int32_t* precs,
                                  int32_t* nb);

/* The bucket layout of a prepared kernel set: up to max_nb buckets into the host arrays cuts,
 * blocks, parts and their number, at most max_nb, into *nb (0 when not prepared); any of the
 * four may be NULL (a tensor-core bucket reports its tile layout in blocks and parts).
 * RF_EINVAL if kern is NULL or max_nb < 0. */
rf_status rf_kernels_os_buckets(const rf_kernels* kern, int32_t max_nb, int32_t* cuts, int32_t* blocks,
                                int32_t* parts, int32_t* nb);

/* Copy the packed taps (sum(len) entries, grid dtype: complex, or real for a real-form set)
 * into caller device memory `dst`.  Async on stream. */
rf_status rf_kernels_copy_taps(const rf_kernels* kern, void* dst, rf_stream stream);

/* Tensor-core layout a kernel set was last prepared for (by its last RF_ALGO_GEMM call): out[0]
 * = rf_prec, out[1] = neighbours per group, out[2] = output tiles of 128 stacked along N,
 * out[3] = taps per K chunk, out[4] = K chunks, out[5] = padded kernel length (all 0 when not
 * prepared).  out is a host int32[6].  RF_EINVAL if kern or out is NULL. */
rf_status rf_kernels_gemm_layout(const rf_kernels* kern, int32_t* out);

/* Borrowed view of the build grid of each kernel (host int64[k]; n for imported kernels). */
rf_status rf_kernels_grids(const rf_kernels* kern, const int64_t** grids);

/* Streaming over data longer than one segment.  With guard = guard_samples, segments of the
 * context's n samples start at s_q = q hop - guard, hop = n - 2 guard (data outside [0, total)
 * taken as zero), so their
 * interiors [s_q + guard, s_q + n - guard) tile the stream; per segment the stored-filter
 * matched filter of the G references (rf_mf_filtered with filt), their window peaks
 * (rf_winmax) and the batched reconstruction of the neighbours (rf_reconstruct_batched,
 * RF_ALGO_AUTO) run on `stream`, and every window of W samples is taken from the segment whose
 * interior holds it.  A segment's circular wrap reaches only its first and last guard samples
 * when guard covers the longest template (its duration from f_low) plus the kernels' lag
 * extents.  x_host: host real[total] (grid dtype); filt: device complex[G][n/2+1] from
 * rf_reference_filters; ks: the G kernel sets.  Outputs (host, caller-owned, nwt = total / W
 * windows; samples past nwt W are not reported): ref_max/ref_arg [G][nwt], nbr_max/nbr_arg
 * [sum k][nwt] (rows as in rf_reconstruct_batched), argmax as int64 stream sample indices.
 * W must divide n and guard, 0 <= 2 guard < n, total >= W.  The context keeps its device and
 * pinned staging buffers between calls (grown on first use); the next segment's upload and the
 * previous segment's host scatter overlap the current segment's work; returns when the stream
 * is done. */
rf_status rf_stream_winmax(rf_ctx* ctx, const void* x_host, int64_t total, int32_t G, const void* filt,
                           rf_kernels* const* ks, int64_t W, int64_t guard_samples, float* ref_max,
                           int64_t* ref_arg, float* nbr_max, int64_t* nbr_arg, rf_stream stream);

/* Template-bank structuring (Sec. III.A), on the host: no context and no device work.
 * Durations tau = -t(f_low) of the stationary-phase templates (t(f) = Psi'(f) / (2 pi) with
 * t_c = 0, Eq. A2, at pn_order).  The bank in chirp-mass order (mc = (m1 m2)^(3/5) /
 * (m1 + m2)^(1/5), ties in bank order) is halved (first half = floor of half) until every
 * set's max tau - min tau <= max_spread (s); each set in symmetric-mass-ratio order (ties in
 * bank order) is halved until it holds at most max_size templates; each set's reference is
 * the template minimising sum_j |tau_i - tau_j| (sums within 1e-9 relative tie; the lowest
 * bank index wins).  Sets are numbered depth first, first half first.
 * bank: host rf_template[count]; outputs (host, caller-owned): set_of[count] (set of each
 * template), ref_of_set[count] (bank index of each set's reference, the first *n_sets
 * entries written), *n_sets, and duration_out[count] (tau, s; may be NULL).  RF_EINVAL for
 * NULL pointers (count > 0), count < 0, f_low <= 0, pn_order outside 0..7, max_spread <= 0 or
 * not finite, max_size < 1. */
rf_status rf_bank_structure(const rf_template* bank, int32_t count, double f_low, int32_t pn_order,
                            double max_spread, int32_t max_size, int32_t* set_of, int32_t* ref_of_set,
                            int32_t* n_sets, double* duration_out);

/* Release a kernel set.  NULL is a no-op. */
void rf_kernels_free(rf_kernels* kern);

/* Neighbour SNR series (Eq. 8, circular):  z_j[i] = sum_{l<L_j} c_j[l] z_ref[(i - m0_j - l) mod n].
 * z_ref: complex[n]; z_out: complex[k][n] (grid dtype).  algo: rf_algo.  RF_ALGO_OS needs an
 * RF_F32 grid with n >= 512 (else RF_EUNSUPPORTED) and evaluates the same sum through the
 * frequency form (Eq. 7) in overlap-save blocks; RF_ALGO_AUTO takes OS on RF_F32 grids and the
 * direct sum on RF_F64 grids.  The context's workspace grows on first use ((B / Lp) n
 * complex64 for OS; see rf_reserve).  Async on stream, except that an OS call on a kernel set that was not
 * prepared prepares it first (see rf_kernels_prepare). */
rf_status rf_reconstruct(rf_ctx* ctx, const void* z_ref, const rf_kernels* kern, int32_t algo,
                         int32_t prec, void* z_out, rf_stream stream);

/* Fused form: per neighbour j and window w of W samples (the last may be short),
 *   max_out[j][w] = max_{wW <= i < (w+1)W} |z_j[i]|^2 (float),
 *   argmax_out[j][w] = the smallest such i (int32, absolute sample index).
 * The full series is never written to memory.  Async on stream. */
rf_status rf_reconstruct_winmax(rf_ctx* ctx, const void* z_ref, const rf_kernels* kern,
                                int32_t algo, int32_t prec, int64_t W, float* max_out,
                                int32_t* argmax_out, rf_stream stream);

/* Batched fused form for G references, each with its own neighbours (Sec. III.A: groups
 * are independent): per reference g, z_refs[g] is its z_ref (device complex[n]) and ks[g]
 * its kernel set; the rows of max_out/argmax_out ([sum_g k_g][ceil(n/W)]) follow the order
 * of the groups and, inside a group, of its neighbours.  algo and prec as in
 * rf_reconstruct_winmax, one choice for all groups.  Overlap-save (AUTO on an RF_F32 grid
 * with n >= 512, or RF_ALGO_OS) runs as one persistent launch over (neighbour, output-block
 * chunk) work units; the direct and tensor-core forms run group after group, each writing
 * its rows in place.  z_refs and ks are host arrays.  For overlap-save, the first
 * call with a given set of references and kernel sets (or after any of them is re-prepared)
 * builds and uploads the work list and allocates the per-reference segment spectra
 * (G x 2n complex64) and window keys, synchronously; later calls with the same arguments
 * only enqueue kernels, so a warmed-up call can be captured in a CUDA graph.  Kernel sets
 * that are not prepared for overlap-save are prepared first.  Async on stream otherwise. */
rf_status rf_reconstruct_batched(rf_ctx* ctx, int32_t G, const void* const* z_refs, rf_kernels* const* ks,
                                 int32_t algo, int32_t prec, int64_t W, float* max_out,
                                 int32_t* argmax_out, rf_stream stream);

/* Autotuner flags. */
enum { RF_TUNE_ALLOW_SPLIT = 1 }; /* the tensor-core form (bf16x6, error about 3e-7 of max|z|) may
                                     be chosen; without it only exact-arithmetic forms compete */

/* One timed candidate of rf_autotune: form (rf_algo), precision (rf_prec) and shape of the
 * kernels shorter than `cut` taps (overlap-save, single-pass or two-phase: block size and
 * partition length; tensor-core form: neighbours per group and stacked output tiles, 0 and 0 for
 * the library's rule; direct sum: 0 and 0), and the form algo2 (RF_ALGO_OS or RF_ALGO_OS_BINS)
 * with block size block2 and partition length part2 of the others (cut = block2 = part2 = algo2
 * = 0: one form and shape for all), and the best of three timings (ms) of the fused window-peak
 * reconstruction of the whole batch. */
typedef struct {
  int32_t algo, block, part, prec, cut, block2, part2, algo2;
  int32_t cut3, block3, part3, algo3; /* a third bucket from cut3 taps on (all 0: none) */
  float ms;
} rf_tune_entry;

/* Autotuner for a batch of G references (z_refs[g], kernel sets ks[g], windows of W samples):
 * times candidate forms on the device and records the fastest in every kernel set, so that
 * RF_ALGO_AUTO uses it from then on (with its precision when it is the tensor-core form).
 * Candidates: on RF_F32 grids the max_os overlap-save layouts of least modelled cost (the batch
 * runs them as in rf_reconstruct_batched) and two-bucket variants (kernels shorter than 2048,
 * 4096 or 8192 taps with one of the two layouts of least modelled cost for them, the others with
 * the fastest single layout), the tensor-core form at RF_PREC_BF16X6 in both tile layouts when
 * flags has RF_TUNE_ALLOW_SPLIT and the mean kernel length is at most 4096 taps, with that flag
 * also the mixed form (the tensor-core form for the shortest eighth of the kernels, up to a
 * power-of-two cut of at most 4096 taps, the fastest single layout for the rest;
 * rf_kernels_prepare_forms), the two-phase form (RF_ALGO_OS_BINS) at the fastest single layout,
 * as the upper bucket of every two-bucket candidate whose layout it takes, and as a third bucket
 * for the kernels of at least 4, 8 or 16 partitions above such a candidate's two, and the direct sum when the grid is RF_F64 or no kernel is longer
 * than 1024 taps.  out (host, may be NULL): up to max_out entries, the winner first; *n_out (host,
 * may be NULL) the number written.  Kernel sets end up prepared for the winner (a bucketed
 * winner, overlap-save or mixed, is then what RF_ALGO_AUTO runs; for another form, the last
 * layout timed).  Allocates; SYNCHRONISES `stream`. */
rf_status rf_autotune(rf_ctx* ctx, int32_t G, const void* const* z_refs, rf_kernels* const* ks, int64_t W,
                      int32_t flags, int32_t max_os, rf_tune_entry* out, int32_t max_out, int32_t* n_out,
                      rf_stream stream);

/* Device-side status of the context: waits for the device, then returns RF_OK, or
 * RF_ETIMEOUT if a bounded device-side wait of an earlier call ran out (that call's outputs
 * are then incomplete), and clears it. */
rf_status rf_device_status(rf_ctx* ctx);

/* Health check of the timeout path (the paper has no counterpart): launches one small kernel
 * that waits, with a short iteration limit, on a barrier nothing arrives on, and records
 * RF_ETIMEOUT in the context's status word as a timed-out tensor-core wait does.  The next
 * rf_device_status then returns RF_ETIMEOUT and clears it; the context stays usable.  Async
 * on stream. */
rf_status rf_selftest_bounded_wait(rf_ctx* ctx, rf_stream stream);

/* Window peaks of `count` series already in memory (e.g. z_ref itself): z: complex[count][n];
 * max_out/argmax_out: [count][ceil(n/W)], same definition as rf_reconstruct_winmax. */
rf_status rf_winmax(rf_ctx* ctx, const void* z, int32_t count, int64_t W, float* max_out,
                    int32_t* argmax_out, rf_stream stream);

/* Reference matched filter without any device allocation.
 *
 * The paper has no counterpart to this call; it exists for callers that cannot call
 * cudaMalloc: for example a plug-in whose host application owns all device memory
 * through its own pool, or a low-latency loop that must not pay for (or synchronise
 * the device on) an allocation.  Such a caller cannot create an rf_ctx, because
 * rf_create allocates the FFT tables and workspaces.
 *
 * It computes what rf_mf_reference computes for one reference template (same
 * arguments, nref = 1, grid passed by value instead of a context) and allocates
 * nothing: no cudaMalloc, no cudaFree, no allocating library routine.  Its
 * workspace is a static device array of about 4 MiB compiled into librf.so, which
 * every GPU that loads the library keeps until the process exits.  That bounds the
 * segment: grid->n must be a power of two in [2^8, 2^16]; larger n returns RF_EINVAL
 * with a message and launches nothing.
 *
 * The array has its own device address in every CUDA context that loads the
 * library: the runtime's primary context of each device, and any context a host
 * application created itself with the driver API and made current.  The first call
 * made in a context looks up that context's address (cudaGetSymbolAddress) and
 * remembers it under the context's process-unique ID (cuCtxGetId), so a later context
 * never receives an earlier one's address, even after cudaDeviceReset; make that first
 * call in each context before any stream capture.  A thread with no current context
 * uses the primary context of its current device.  All calls share the one workspace and it keeps the
 * last call's contents; every call rewrites each part it reads, so results never
 * depend on an earlier call.  Calls whose work overlaps on the GPU (different
 * streams, or different host threads) race on the workspace and corrupt each other:
 * serialise them, e.g. on one stream.
 *
 * x, inv_psd, z_out (complex[n]) and sigma_out (double[1], may be NULL) are caller
 * device memory, 16-byte aligned; ref is host memory.  Async on stream. */
rf_status rf_mf_reference_noalloc(const rf_grid* grid, const void* x, const double* inv_psd,
                                  const rf_template* ref, void* z_out, double* sigma_out,
                                  rf_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* RF_H */
