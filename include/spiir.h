/*
 * spiir.h -- C ABI of the B300 (sm_103a) SPIIR hot path.
 *
 * The library computes the data-parallel part of the SPIIR coherent search
 * (arxiv 2011.06787): whitened multi-detector strain -> bank of complex first-order
 * IIR filters -> complex SNR per template and detector -> coherent all-sky scan ->
 * maximum network statistic, its sky pixel and the null stream.
 *
 * Conventions shared by every entry point
 *   - Return value: SPIIR_OK (0) or a negative SPIIR_E* code.  spiir_last_error()
 *     returns a text description of the last failure on the calling thread.  No C++
 *     exception crosses this interface and nothing aborts the process.
 *   - Pointers named *_dev are CUDA device pointers on the current device; *_host are
 *     host pointers.  The caller owns every buffer it passes; the library owns the
 *     objects it creates (banks, sky tables, pipelines) and everything inside them.
 *   - Complex values are interleaved (re, im) float pairs.  Sizes are in elements.
 *   - stream is a cudaStream_t passed as void* (NULL = legacy default stream).  Work is
 *     enqueued asynchronously on it unless the entry point says otherwise.
 *   - Arguments are validated on the host before anything is launched; a rejected call
 *     leaves every object unchanged.
 *   - Kernels never trap.  A device-side wait that runs out of iterations sets a sticky
 *     error word that spiir_device_status() reports (SPIIR_ETIMEOUT).
 */
#ifndef SPIIR_H
#define SPIIR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SPIIR_OK 0
#define SPIIR_EINVAL (-1)       /* invalid argument (shape, range, non-finite value, NULL) */
#define SPIIR_ECUDA (-2)        /* a CUDA runtime call failed */
#define SPIIR_ENOMEM (-3)       /* host or device allocation failed */
#define SPIIR_EUNSUPPORTED (-4) /* valid input outside what this build supports */
#define SPIIR_ETIMEOUT (-5)     /* a bounded device-side wait gave up */

typedef struct spiir_bank_s *spiir_bank_t;
typedef struct spiir_sky_s *spiir_sky_t;
typedef struct spiir_pipeline_s *spiir_pipeline_t;
typedef struct spiir_batch_s *spiir_batch_t;
typedef struct spiir_frontend_s *spiir_frontend_t;
typedef struct spiir_search_s *spiir_search_t;

/* Library version (major * 10000 + minor * 100 + patch). */
int spiir_version(void);

/* Copy the last error message of the calling thread into buf (NUL-terminated,
 * truncated to len).  Returns the full message length. */
int spiir_last_error(char *buf, size_t len);

/* Test hook: make the next n allocations made by the library fail with SPIIR_ENOMEM
 * (0 disables).  Used to exercise allocation-failure paths without a real shortage. */
void spiir_debug_fail_allocs(int n);

/* Test hook: only the k-th device or pinned-host allocation from now fails (k >= 1; 0
 * disarms), so that the clean-up of a partially built object can be exercised at every
 * allocation site.  No counterpart in the paper. */
void spiir_debug_fail_alloc_at(int k);

/* Test hook for failure detection, with no counterpart in the paper: launches one block on
 * `stream` whose bounded wait on an mbarrier that nothing completes gives up after
 * `iterations` tries (1 .. 2^26) and records a timeout in the device status word, as a
 * production wait that ran out does.  The next spiir_device_status call reports
 * SPIIR_ETIMEOUT; the context stays usable.  Errors: SPIIR_EINVAL, SPIIR_ECUDA. */
int spiir_debug_wait_timeout(uint32_t iterations, void *stream);

/* Sticky device-side status: SPIIR_OK, or SPIIR_ETIMEOUT after a bounded wait inside a
 * kernel gave up.  Synchronises the device.  clear != 0 resets the word.  The word is a
 * file-scope device variable: neither this call nor any kernel allocates it. */
int spiir_device_status(int clear);

/* ------------------------------------------------------------------------------------
 * Filter bank -- Sec. II.B.1, Eq. (zk), read per filter (the commented closed form
 * u(t) = sum_m b_m a_m^(t - t_m) beside it fixes that reading):
 *     y_l[k] = a1_l * y_l[k-1] + b0_l * x_I[k - d_l]
 *     z_{t,I}[k] = sum_{l in template t} y_l[k]
 * for every detector I.  12 flops per filter per sample (Sec. II.B.2).
 * ---------------------------------------------------------------------------------- */

/* Create a bank of n_templates templates for a network of n_det detectors.
 *   filter_offsets_host [n_templates + 1]  CSR offsets; template t owns filters
 *                                          [off[t], off[t+1]); off[0] = 0.
 *   a1_host [2 F]   feedback coefficients (re, im), |a1| < 1 required (stability; the
 *                   paper does not state the bound).
 *   b0_host [2 F]   feedforward coefficients (re, im), finite.
 *   delay_host [F]  integer delays d_l in samples, 0 <= d_l <= 1<<20.
 * The coefficients are copied; the bank owns its IIR states (all zero) and a strain
 * history of max(d_l) samples per detector (zero).  A bank whose largest delay is at least
 * 16384 samples is cut into delay bins of 8192 samples with 256-lane blocks (see
 * spiir_bank_set_delay_bin), so long templates (a 74 s chirp from 30 Hz spans about 151k
 * samples at 2048 Hz) fit.
 * Errors: SPIIR_EINVAL for bad shapes or values, SPIIR_EUNSUPPORTED when one template has
 * more filters than one thread block can hold (4096 in this build), SPIIR_ENOMEM,
 * SPIIR_ECUDA. */
int spiir_bank_create(int n_det, int n_templates, const int64_t *filter_offsets_host,
                      const float *a1_host, const float *b0_host, const int32_t *delay_host,
                      spiir_bank_t *out);
void spiir_bank_destroy(spiir_bank_t bank);

/* Shape query.  Any output pointer may be NULL. */
int spiir_bank_info(spiir_bank_t bank, int *n_det, int *n_templates, int64_t *n_filters,
                    int32_t *max_delay);

/* Zero the IIR states and the strain history (start of a new stream).  Enqueued on
 * stream. */
int spiir_bank_reset(spiir_bank_t bank, void *stream);

/* Checkpoint / resume of the streaming state.  The state is the IIR state y_l of every
 * filter and detector plus the last max(d_l) strain samples per detector, serialised
 * in the caller's filter order.  spiir_bank_state_bytes gives the size.  get/set
 * synchronise the device; set_state rejects a buffer of the wrong size or of another
 * bank shape (SPIIR_EINVAL). */
int spiir_bank_state_bytes(spiir_bank_t bank, size_t *bytes);
int spiir_bank_get_state(spiir_bank_t bank, void *host, size_t bytes);
int spiir_bank_set_state(spiir_bank_t bank, const void *host, size_t bytes);

/* Launch shape of the filter-bank kernel, a tuning knob: the filtered values do not depend on
 * it beyond the order of floating-point summation.  filters_per_lane in {4, 8, 16},
 * lanes_per_block in {128, 256}, steps_per_reduce in {16, 20, 32, 64}, tile a multiple of
 * steps_per_reduce up to 8192 (samples per staged strain window).  The streaming state is
 * kept.  Synchronises the device.  SPIIR_EUNSUPPORTED if a template does not fit or the
 * window does not fit in shared memory; the bank then keeps its previous shape.
 * Defaults: 8, 128, 32, 1024; 256 lanes when a template exceeds 1024 filters and 16
 * filters per lane when it exceeds 2048. */
int spiir_bank_set_shape(spiir_bank_t bank, int filters_per_lane, int lanes_per_block,
                         int steps_per_reduce, int tile);
int spiir_bank_get_shape(spiir_bank_t bank, int *filters_per_lane, int *lanes_per_block,
                         int *steps_per_reduce, int *tile);

/* Delay bins (a layout knob for long templates; results do not depend on it beyond the order
 * of floating-point summation).  Each thread block stages one strain window per time tile that
 * covers the delays of its own filters.  With delay_bin = B > 0 the filters of template t whose
 * delays lie in [jB, (j+1)B) form piece j of t; blocks hold pieces of one bin only, so a
 * window spans at most B + tile samples.  A template's first piece writes its SNR row, its
 * later pieces write rows of a bank-owned buffer that one more launch adds into the SNR, in
 * bin order: z_t = sum_j z_t^(j).  delay_bin = 0 keeps every template whole (one window of the
 * bank's largest delay).  B is 0 or a multiple of 4 in [1024, 1<<20].  Keeps the streaming
 * state; synchronises the device.  Default: 0 below a largest delay of 16384, else 8192.
 * get: the bin width, the number of thread blocks and of pieces (templates + extra pieces).
 * Errors: SPIIR_EINVAL; SPIIR_EUNSUPPORTED when a window does not fit in shared memory (the
 * bank keeps its previous layout). */
int spiir_bank_set_delay_bin(spiir_bank_t bank, int32_t delay_bin);
int spiir_bank_get_delay_bin(spiir_bank_t bank, int32_t *delay_bin, int *n_blocks, int *n_pieces);

/* Filter one chunk of strain and advance the streaming state.
 *   strain_dev [n_det][strain_pitch] float; samples 0..n-1 of each row are this chunk,
 *              continuing the stream seen by previous calls.
 *   snr_dev    [n_templates][n_det][snr_pitch] complex (2 floats); sample k of the
 *              chunk is written at index k of each row; other entries are untouched.
 * n >= 1, strain_pitch >= n, snr_pitch >= n.  Enqueued on stream.  Calls on the same
 * bank must be ordered (one stream, or explicit synchronisation). */
int spiir_filter_chunk(spiir_bank_t bank, const float *strain_dev, int64_t strain_pitch,
                       int64_t n, float *snr_dev, int64_t snr_pitch, void *stream);

/* Filter one segment that starts a stream without allocating anything -- for callers that
 * cannot call cudaMalloc (for example code running where device allocation is forbidden or
 * would stall, or under an allocator that owns all device memory).  The paper has no
 * counterpart; this is a packaging of the filter bank above.
 * Computes what spiir_bank_create followed by one spiir_filter_chunk computes on a new bank
 * (zero IIR states, zero strain history), with the same kernel.  Coefficient arguments are
 * host arrays as in spiir_bank_create; strain_dev and snr_dev are as in spiir_filter_chunk.
 * All scratch (copied coefficients, packed layout, block tables, IIR states, strain window)
 * lives in one file-scope device array of 32 MiB that every GPU which loads the library
 * holds until the process exits; no cudaMalloc, cudaFree or other allocating routine is
 * called.  The first call on a device looks up that array's device address with the device
 * current (cudaGetSymbolAddress), so make the first call before any stream capture.
 * Every call reuses the same array: calls whose GPU work can overlap (different streams
 * without ordering) race and give wrong results; order them on one stream.  Everything,
 * including the copies of the host arrays into the array, is enqueued on stream: the host
 * arrays must stay valid and unchanged until the stream has passed this call (for example,
 * until cudaStreamSynchronize(stream) returns).  A bounded device wait that runs out is
 * reported by spiir_device_status, as for every other kernel of the library.
 * Limits: n_det <= 4, n_templates <= 4096, n_filters <= 131072, n <= 65536, delays <= 8192,
 * and the packed problem must fit in the array; otherwise SPIIR_EUNSUPPORTED with the limit
 * in spiir_last_error().  Invalid values: SPIIR_EINVAL as in spiir_bank_create. */
int spiir_filter_static(int n_det, int n_templates, const int64_t *filter_offsets_host,
                        const float *a1_host, const float *b0_host, const int32_t *delay_host,
                        const float *strain_dev, int64_t strain_pitch, int64_t n, float *snr_dev,
                        int64_t snr_pitch, void *stream);

/* ------------------------------------------------------------------------------------
 * Sky tables -- Sec. II.C.1 (HEALPix tiling, U and time-offset look-up tables) and
 * App. A Eqs. (strain_sngl), (svd).
 * ---------------------------------------------------------------------------------- */

/* Host-side FP64 construction of the per-pixel tables for one epoch (no Earth
 * rotation) from detector geometry, stored as int32 / FP32.
 *   det_pos_m [n_det][3]  Earth-fixed detector positions (m)
 *   arm_x, arm_y [n_det][3] unit arm directions
 *   sigma [n_det]          noise weights sigma_I (App. A Eq. (h_prop))
 *   nside                  HEALPix resolution; n_pix = 12 nside^2, RING order
 *   rate_hz                sample rate of the SNR series
 * Outputs (caller-allocated host arrays):
 *   delays [n_pix][n_det]   Delta_I(p) = round(-rate * nhat_p . r_I / c), half away from
 *                           zero: detector I's SNR for geocentric sample k is read at
 *                           k + Delta_I(p).
 *   u_sig  [n_pix][n_det][2]          first two columns of U in G_sigma = U Lambda V^T
 *   u_null [n_pix][n_det][n_det - 2] remaining columns (may be NULL when n_det = 2)
 * 2 <= n_det <= 4, 1 <= nside <= 64.  A pixel whose G_sigma has sigma_2 / sigma_1 <
 * 1e-6 gets a zero second signal column (projection onto the numerical rank). */
int spiir_sky_tables(int n_det, const double *det_pos_m, const double *arm_x,
                     const double *arm_y, const double *sigma, int nside, double rate_hz,
                     int32_t *delays, float *u_sig, float *u_null);

/* Upload per-pixel tables (layouts as produced by spiir_sky_tables) to the device.
 * The halo H = max |delays| sets the SNR padding that spiir_coherent_scan needs.
 * |delays| <= 1024.  Errors: SPIIR_EINVAL, SPIIR_ENOMEM, SPIIR_ECUDA. */
int spiir_sky_create(int n_det, int n_pix, const int32_t *delays_host, const float *u_sig_host,
                     const float *u_null_host, spiir_sky_t *out);
void spiir_sky_destroy(spiir_sky_t sky);
int spiir_sky_info(spiir_sky_t sky, int *n_det, int *n_pix, int *halo);

/* Launch shape of the coherent scan for 2 and 3 detectors, a tuning knob that does not change
 * results: threads per block in {256, 512}, pairs of output samples per thread in {1, 2}, and
 * table_in_shared 1 to keep the pixel table in shared memory when it fits (0 reads it through
 * the L1 cache and leaves the shared memory to more resident blocks).  Synchronises the
 * device.  grouped (output) is 1 when the grouped scan applies: 2 or 3 detectors, an
 * orthonormal U with a rank-2 signal plane, at most 65535 pixels.  Default 256 threads,
 * 2 pairs, table in shared memory.
 * pairs = 4 selects the tensor-memory scan (3 detectors, pixel table within shared memory):
 * each of 128 thread rows keeps the detector-1 and -2 SNR windows of its consecutive samples
 * in tensor memory (one block per SM, 512 columns); threads = 512 gives 8 samples per row
 * (max |Delta| <= 60), threads = 256 gives 16 (max |Delta| <= 56, whole 2048-sample chunks per
 * work item, fewer per-pixel overheads per sample with half the warps).  Both pair the FP32
 * arithmetic differently from the shared-memory scan, so they agree with it to rounding and
 * with each other bit for bit; with a sky map each thread writes its samples of a pixel as
 * one contiguous segment.
 * For this shape the third value selects where the pixel groups and per-pixel delay offsets
 * are read: 1 (default) from the kernel's parameter space (warp-uniform reads, so the
 * tensor-memory addresses stay in uniform registers), 0 from shared memory.  A sky above 6400
 * pixels or 256 pixel groups is scanned as the fewest consecutive parts of nearly equal pixel
 * counts within those limits (two at nside 32), one launch each, with the same results.
 * Errors: SPIIR_EUNSUPPORTED when the tensor-memory scan does not apply (the previous shape is
 * kept), SPIIR_EINVAL for other shapes. */
int spiir_sky_set_scan_shape(spiir_sky_t sky, int threads, int pairs, int table_in_shared);
int spiir_sky_get_scan_shape(spiir_sky_t sky, int *threads, int *pairs, int *table_in_shared,
                             int *grouped);

/* Coherent all-sky scan -- Sec. II.C.1 Eq. (llr_form) and Eq. (null_def), App. A:
 *     w_I(p, k)   = z_I[k + Delta_I(p)]
 *     rho_C^2(p,k) = sum_{j=1,2} | sum_I U_s[p][I][j] w_I |^2
 *     max_stat[k] = max_p rho_C^2(p, k), argmax[k] = lowest p attaining it
 *     null_stat[k] = sum_{j>2} | sum_I U_null[p][I][j] w_I |^2 at p = argmax[k]
 *                    (0 when n_det = 2)
 *   snr_dev [n_templates][n_det][snr_pitch] complex; entry H + j of a row holds the
 *           SNR of output sample j (H = halo), so rows need snr_pitch >= n + 2 H.
 *   max_stat_dev, null_stat_dev [n_templates][n] float; argmax_dev [n_templates][n] int32.
 *   skymap_dev  NULL, or [n_templates][n_pix][n] float receiving rho_C^2 of every pixel
 *               (pixel-major so that consecutive samples are contiguous).
 * Enqueued on stream. */
int spiir_coherent_scan(spiir_sky_t sky, const float *snr_dev, int64_t snr_pitch,
                        int n_templates, int64_t n, float *max_stat_dev, int32_t *argmax_dev,
                        float *null_stat_dev, float *skymap_dev, void *stream);

/* ------------------------------------------------------------------------------------
 * Signal-consistency statistic (Sec. II.C.2).  For template t, detector I and sample k,
 *   xi_I^2[k] = sum_{j=-Nj}^{Nj} |z_I[k + j] - z_I[k] A_t[j]|^2 / sum_{j=-Nj}^{Nj} (2 - 2 |A_t[j]|^2)
 * with A_t the autocorrelation of the template's response u_t (A[j] = R[j] / R[0],
 * R[j] = sum_k conj(u[k]) u[k + j], A[-j] = conj(A[j])); the SNR is taken as normalised
 * (E|z|^2 = 2 in noise), so the statistic is a reduced chi-square of mean 1.  The network
 * value is xi_C^2 = (1 / N_d) sum_I xi_I^2, each detector read at its arrival time for the
 * coherent argmax pixel.  Nj ("n_lags") is typically 175 (Sec. III.D); at most 1024.
 * ---------------------------------------------------------------------------------- */

/* A_dev [T][2 n_lags + 1] complex (entry n_lags + j is lag j) from the responses
 * u_dev [T][n_resp] complex (e.g. spiir_impulse_forward with zero initial states); lags past
 * the response contribute nothing.  Device pointers, enqueued on stream.
 * Errors: SPIIR_EINVAL. */
int spiir_autocorr(int n_templates, const float *u_dev, int64_t n_resp, int n_lags, float *A_dev,
                   void *stream);

/* xi2_dev [T][n_det][xi2_pitch] (f32): xi_I^2 of samples k = 0 .. n-1, from
 * snr_dev [T][n_det][snr_pitch] complex in which entry n_lags + k is sample k (samples
 * -n_lags .. n + n_lags - 1 are read; snr_pitch >= n + 2 n_lags, 8-byte aligned) and
 * A_dev [T][2 n_lags + 1] complex.  Device pointers, enqueued on stream.
 * Errors: SPIIR_EINVAL. */
int spiir_xi2(int n_templates, int n_det, const float *snr_dev, int64_t snr_pitch, const float *A_dev,
              int n_lags, int64_t n, float *xi2_dev, int64_t xi2_pitch, void *stream);

/* out_dev [T][n] (f32): xi_C^2 at every (template, sample) of a coherent scan of the same SNR,
 * from xi2_dev [T][n_det][xi2_pitch] in which entry H + k is sample k (H = the sky's halo,
 * xi2_pitch >= n + 2 H) and argmax_dev [T][n] (the scan's argmax).  An argmax outside the sky
 * gives NaN.  Device pointers, enqueued on stream.  Errors: SPIIR_EINVAL. */
int spiir_xi2_network(spiir_sky_t sky, int n_templates, const float *xi2_dev, int64_t xi2_pitch,
                      const int32_t *argmax_dev, int64_t n, float *out_dev, void *stream);

/* ------------------------------------------------------------------------------------
 * Front end (Sec. II.A): down-sampling and whitening of the strain before the filter bank.
 * Each detector's strain at the input rate (16384 Hz in the paper) is low-passed and
 * decimated by M with a time-domain FIR filter, x_2[j] = sum_{i < L_d} h[i] x[j M - i], then
 * whitened by a causal FIR of its own, y_I[k] = sum_{i < L_w} w_I[i] x_2,I[k - i].  The paper
 * whitens in the frequency domain, Eq. (whiten), dividing by sqrt(S_n(f)); with
 * spiir_whitening_kernel the FIR has that response (scaled to unit-variance output) with linear
 * phase, so the output lags by (L_w - 1) / 2 samples and needs no segment collection.  The
 * decimation filter's own delay (L_d - 1) / 2 input samples is not compensated either.
 * ---------------------------------------------------------------------------------- */

/* Host helper: Hann-windowed sinc low-pass for decimation by M with cutoff
 * cutoff x (output Nyquist frequency), 0 < cutoff <= 1, unit DC gain, designed in FP64:
 * h[i] = 2 fc sinc(2 fc (i - (n-1)/2)) (1/2 - 1/2 cos(2 pi (i + 1/2) / n)) / sum, fc = cutoff / (2 M)
 * cycles per input sample.  taps_host [n_taps], n_taps <= 8192, M <= 64.  Errors: SPIIR_EINVAL. */
int spiir_fir_lowpass(int n_taps, int M, double cutoff, float *taps_host);

/* Host helper: whitening FIR of Eq. (whiten) from a one-sided PSD.  psd_host[j] is S_n at
 * f_j = j rate_hz / N, j = 0 .. n_freq - 1, N = 2 (n_freq - 1), each finite and > 0.  With
 * A_j = sqrt(2 / (rate_hz S_n(f_j))), the zero-phase response on the N-point grid has the
 * impulse response a[m] = (1/N) [A_0 + (-1)^m A_{N/2} + 2 sum_{0<j<N/2} A_j cos(2 pi j m / N)];
 * taps_host[i] = win[i] a[i - K] for i < n_taps = 2K + 1 (odd, below N, at most 16385), with
 * the Hann window win[i] = 1/2 - 1/2 cos(2 pi (i + 1) / (n_taps + 1)).  Noise of PSD S_n comes
 * out with unit variance.  FP64 design, FP32 taps.  Errors: SPIIR_EINVAL. */
int spiir_whitening_kernel(int n_freq, const double *psd_host, double rate_hz, int n_taps,
                           float *taps_host);

/* Streaming front end for n_det detectors: the decimation taps (shared by all detectors) and
 * one whitening kernel per detector (white_taps_host [n_det][n_white_taps]) are copied to the
 * device; the FIR histories are owned by the object and start at zero.  max_in: the largest
 * input segment (a multiple of M).  n_dec_taps <= 8192, n_white_taps <= 16385, M <= 64.
 * Errors: SPIIR_EINVAL, SPIIR_ENOMEM, SPIIR_ECUDA. */
int spiir_frontend_create(int n_det, int M, int n_dec_taps, const float *dec_taps_host,
                          int n_white_taps, const float *white_taps_host, int64_t max_in,
                          spiir_frontend_t *out);
void spiir_frontend_destroy(spiir_frontend_t fe);
/* Shape query: detectors, decimation factor and the largest input segment.  Any output
 * pointer may be NULL. */
int spiir_frontend_info(spiir_frontend_t fe, int *n_det, int *M, int64_t *max_in);
/* Zero the histories (a new stream).  Enqueued on stream. */
int spiir_frontend_reset(spiir_frontend_t fe, void *stream);
/* One segment: strain_dev [n_det][strain_pitch] f32 at the input rate, n_in samples (a positive
 * multiple of M, at most max_in); out_dev [n_det][out_pitch] f32 receives the n_in / M
 * whitened samples at the output rate.  Continues the stream of the previous call.  Two
 * launches on stream, the second a programmatic dependent launch of the first.
 * Errors: SPIIR_EINVAL, SPIIR_ECUDA. */
int spiir_frontend_run(spiir_frontend_t fe, const float *strain_dev, int64_t strain_pitch,
                       int64_t n_in, float *out_dev, int64_t out_pitch, void *stream);

/* ------------------------------------------------------------------------------------
 * Candidates and the time-shift background (Sec. II.C.1, II.C.3).
 * A single-detector candidate is a sample k of detector I at which the largest |z_I| over
 * the bank's templates exceeds the threshold (4 in the paper); it belongs to the template
 * that attains that maximum (the lowest template among equals), and each template keeps at
 * most one candidate per second: its largest, the earliest among equals.  Seconds are
 * counted from sample 0 of the analysed span in blocks of per_second samples.  Every
 * comparison is made on |z|^2 = re*re + im*im in FP32 with each operation rounded, against
 * threshold^2 rounded the same way, so the selection is exact and reproducible.
 * Each candidate is then evaluated coherently at every sky pixel p: its own detector is read
 * at its sample and every other detector J at k + Delta_J(p) - Delta_I(p) + shift_J, the
 * times a source in direction p implies.  Time shift s moves the c-th other detector of I
 * (c = 1, 2, ... in detector order) by shift_J = -s c step samples (it is read earlier);
 * s = 0 is the zero-lag (foreground) statistic, s = 1..100 with step = 205 (0.1 s at
 * 2048 Hz) the paper's background.
 * ---------------------------------------------------------------------------------- */

/* Bytes of the workspace spiir_select_candidates needs: one 64-bit slot per
 * (detector, template, second), one 64-bit key per (detector, sample) and one 64-bit word
 * for a block counter.  Errors: SPIIR_EINVAL. */
int spiir_select_workspace_bytes(int n_templates, int n_det, int64_t n, int per_second,
                                 size_t *bytes);

/* Select the candidates of samples 0 .. n-1 of snr_dev [T][n_det][snr_pitch] complex, in
 * which entry snr_offset + k is sample k (snr_offset + n <= snr_pitch; n_det n and
 * n_det T seconds below 2^31).
 *   workspace_dev: device buffer of at least spiir_select_workspace_bytes, 8-byte aligned,
 *       ALL ZERO on entry (cudaMemset once after allocation); the call leaves it zero.
 *   cand_dev [max_cand][4] int32, 16-byte aligned: (detector, template, sample, bits of the
 *       FP32 |z|^2) ordered by detector, then template, then second.
 *   n_cand_dev: one int32 on the device, set to the number of candidates found (records past
 *       max_cand are dropped: a count above max_cand signals the overflow).
 * Two launches on stream, the second a programmatic dependent launch of the first (it may
 * be scheduled early and waits for the first to complete); nothing is synchronised and
 * nothing returns to the host.  The threshold must be finite and >= 0.  NaN SNR values are
 * never candidates.
 * Errors: SPIIR_EINVAL. */
int spiir_select_candidates(int n_templates, int n_det, const float *snr_dev, int64_t snr_pitch,
                            int64_t snr_offset, int64_t n, float threshold, int per_second,
                            void *workspace_dev, size_t workspace_bytes, int32_t *cand_dev,
                            int max_cand, int32_t *n_cand_dev, void *stream);

/* Coherent statistic at the first min(*n_cand_dev, max_cand) candidates of cand_dev (the
 * records of spiir_select_candidates, or any (detector, template, sample, unused) records),
 * under the time shifts s = first_shift .. first_shift + n_shifts - 1 (shift_step samples
 * per unit), on the SNR snr_dev [T][n_det][snr_pitch] in which entry snr_offset + k is
 * sample k.  Outputs [max_cand][n_shifts] (row c, column s - first_shift):
 *   max_dev    max over pixels of rho_C^2 (same U tables and arithmetic as
 *              spiir_coherent_scan), argmax_dev the pixel (lowest among equals),
 *   null_dev   the null stream at that pixel (0 for two detectors).
 * An entry whose reads would leave [0, snr_pitch) for some pixel, or whose record names a
 * detector or template outside the sky or bank, is (NaN, -1, NaN).  Rows past the count are
 * not written.  For the background the SNR must hold first_shift + n_shifts - 1 times
 * (n_det - 1) shift_step samples of history before the earliest candidate, plus the sky's
 * delay range.  One persistent launch on stream, a programmatic dependent launch (it may be
 * scheduled before the stream's previous kernel completes and waits for it before reading);
 * the count is read on the device.
 * Errors: SPIIR_EINVAL, SPIIR_EUNSUPPORTED (SNR windows above 200 KB of shared memory). */
int spiir_coherent_candidates(spiir_sky_t sky, int n_templates, const float *snr_dev,
                              int64_t snr_pitch, int64_t snr_offset, const int32_t *cand_dev,
                              const int32_t *n_cand_dev, int max_cand, int first_shift,
                              int n_shifts, int shift_step, float *max_dev, int32_t *argmax_dev,
                              float *null_dev, void *stream);

/* xi^2 at candidates (Sec. II.C.2 at the points of spiir_coherent_candidates): for the first
 * min(*n_cand_dev, max_cand) records of cand_dev and the shifts s = first_shift ..
 * first_shift + n_shifts - 1, with p = argmax_dev[c][s - first_shift] the coherent argmax of the
 * item (as spiir_coherent_candidates writes it), detector J of the candidate's template is read
 * at x_J = snr_offset + k + Delta_J(p) - Delta_r(p) + shift_J, shift_J = -s c step for the c-th
 * companion of the candidate's detector r (0 for r), and
 *   xi_J^2 = sum_{j=-Nj}^{Nj} |z_J[x_J + j] - z_J[x_J] A_t[j]|^2 / sum_j (2 - 2 |A_t[j]|^2)
 * with A_dev [T][2 n_lags + 1] as in spiir_xi2.  xi2_dev [max_cand][n_shifts] receives
 * (1 / N_d) sum_J xi_J^2; xi2_det_dev, if not NULL, [max_cand][n_shifts][n_det] the
 * per-detector values.  NaN where p is not a pixel of the sky, the record names a detector or
 * template outside the sky or bank, or a read would leave [0, snr_pitch).  Rows past the count
 * are not written.  One persistent launch on stream, a programmatic dependent launch as for
 * spiir_coherent_candidates.  Errors: SPIIR_EINVAL. */
int spiir_xi2_candidates(spiir_sky_t sky, int n_templates, const float *snr_dev, int64_t snr_pitch,
                         int64_t snr_offset, const float *A_dev, int n_lags, const int32_t *cand_dev,
                         const int32_t *n_cand_dev, int max_cand, int first_shift, int n_shifts,
                         int shift_step, const int32_t *argmax_dev, float *xi2_dev,
                         float *xi2_det_dev, void *stream);

/* ------------------------------------------------------------------------------------
 * Candidate-driven streaming search (Sec. II.C.1 - II.C.3): the paper's coherent stage as it
 * runs per chunk.  One call filters a chunk of strain into a ring of SNR history (Sec. II.B.1)
 * and, on the span of the stream that the ring now fully surrounds, selects the
 * single-detector candidates (spiir_select_candidates), evaluates the coherent statistic and
 * null stream at every candidate at zero lag on the foreground sky and under the time shifts
 * 1 .. n_shifts on the background sky (spiir_coherent_candidates), and xi_C^2 at each of those
 * coherent argmax pixels (spiir_xi2_candidates).  The candidate count stays on the device;
 * nothing is synchronised.
 * Span: a call analyses the chunk-long span [S0, S0 + chunk) of stream samples with
 * S0 = (samples filtered after the call) - chunk - La, La = 2 H + n_lags (H the larger sky
 * halo): the search lags the strain by La samples, the most the zero-lag stages read past a
 * candidate.  The background and xi^2 read back up to
 * Hb = n_shifts (n_det - 1) shift_step + 2 H + n_lags samples before a candidate, so the ring
 * keeps L = Hb + chunk + La samples per (template, detector) (2 L entries: each sample is
 * stored twice so that any L consecutive samples are contiguous).  Samples before the stream
 * start are zero.  Seconds (one candidate per template per second) are blocks of per_second
 * samples counted from S0.
 * Overlapped mode (SPIIR_SEARCH_OVERLAP): a call analyses the span that the ring surrounded
 * before the call, S0 = (samples filtered before the call) - chunk - La, on an internal
 * stream, while the filter bank takes the new chunk on the caller's stream; the caller's
 * stream then waits for the candidate stages.  The search lags one chunk more, the ring keeps
 * L = Hb + 2 chunk + La samples, and the first call's span lies before the stream start.
 * ---------------------------------------------------------------------------------- */

#define SPIIR_SEARCH_OVERLAP 1 /* flag of spiir_search_create */

/* bank, sky_fg (zero lag; nside 16 in the paper), sky_bg (time shifts; nside 8) must share
 * n_det >= 2 and outlive the search, and the bank is driven only through it.  A_dev
 * [T][2 n_lags + 1] complex: each template's autocorrelation as for spiir_xi2 (copied).
 * chunk: strain samples per call.  threshold: |z| above which a sample is a candidate (4 in
 * the paper).  n_shifts (100 in the paper, 0 for none) time shifts of shift_step samples per
 * companion (205 = 0.1 s at 2048 Hz).  max_cand: rows of the candidate outputs.  flags: 0 or
 * SPIIR_SEARCH_OVERLAP (the search then owns a CUDA stream and two events on the current
 * device).  Errors: SPIIR_EINVAL, SPIIR_ENOMEM, SPIIR_ECUDA. */
int spiir_search_create(spiir_bank_t bank, spiir_sky_t sky_fg, spiir_sky_t sky_bg, const float *A_dev,
                        int n_lags, int64_t chunk, float threshold, int per_second, int n_shifts,
                        int shift_step, int max_cand, int flags, spiir_search_t *out);
void spiir_search_destroy(spiir_search_t search);
/* Ring length L, history Hb and lag La (samples), and S0 of the next call's span. */
int spiir_search_info(spiir_search_t search, int64_t *ring_len, int64_t *history, int64_t *lag,
                      int64_t *next_span_start);
/* Zero the bank's state and the ring (a new stream).  Enqueued on stream. */
int spiir_search_reset(spiir_search_t search, void *stream);
/* One chunk.  strain_dev [n_det][strain_pitch] f32, chunk samples continuing the stream.
 * Outputs (device, caller-owned; rows past the count are not written):
 *   cand_dev [max_cand][4] int32 (16-byte aligned): (detector, template, sample k of the span,
 *     bits of the FP32 |z|^2) as spiir_select_candidates; stream sample = S0 + k.
 *   n_cand_dev [1] int32: candidates found (above max_cand on overflow).
 *   fg_*_dev [max_cand]: zero-lag maximum of rho_C^2 over the foreground sky, its pixel, the
 *     null stream there and xi_C^2 there.
 *   bg_*_dev [max_cand][n_shifts]: the same for shifts 1 .. n_shifts on the background sky
 *     (may be NULL when n_shifts = 0).
 *   span_start: NULL or a host int64 that receives S0.
 * Calls on one search must be ordered on one stream; in overlapped mode the outputs are
 * written on the internal stream and are complete, in the caller's stream order, after the
 * call's work.  Errors: SPIIR_EINVAL, SPIIR_ECUDA. */
int spiir_search_run(spiir_search_t search, const float *strain_dev, int64_t strain_pitch,
                     int32_t *cand_dev, int32_t *n_cand_dev, float *fg_max_dev,
                     int32_t *fg_argmax_dev, float *fg_null_dev, float *fg_xi2_dev,
                     float *bg_max_dev, int32_t *bg_argmax_dev, float *bg_null_dev,
                     float *bg_xi2_dev, int64_t *span_start, void *stream);

/* ------------------------------------------------------------------------------------
 * Impulse response and its adjoint, for refining IIR coefficients against target
 * templates (the overlap of Sec. II.B.1 Eq. (overlap) is the usual objective).
 * Layout: T templates x F filters each (F <= 1024), row-major [T][F]; complex values are
 * interleaved pairs.  All pointers are device pointers.
 * ---------------------------------------------------------------------------------- */

/* u_t[k] = sum_l y_l[k] for k = 0..n-1, with y_l[-1] = s0_l and
 * y_l[k] = a1_l y_l[k-1] + b0_l [k == d_l] (Eq. (zk) driven by a unit impulse at k = 0).
 *   u_dev [T][n] complex.  ckpt_dev: NULL, or [ceil(n / ckpt_every)][T][F] complex that
 *   receives y_l[j ckpt_every - 1] for every j (the state before sample j ckpt_every);
 *   ckpt_every a multiple of 32 in [32, 8192].  Delays may exceed n.  Enqueued on stream.
 * With checkpoints the segment starting states are found by jumps in double-float (pairs of
 * FP32 numbers, about 44 significant bits; no FP64 runs on the device),
 *   y[(j+1)C - 1] = a^C y[jC - 1] + b a^((j+1)C - 1 - d) [jC <= d < (j+1)C],
 * and the segments run in parallel in FP32; without, one pass per template over all n, which
 * holds at most 864 filters per template (SPIIR_EUNSUPPORTED above). */
int spiir_impulse_forward(int n_templates, int filters_per_template, const float *a1_dev,
                          const float *b0_dev, const int32_t *delay_dev, const float *s0_dev,
                          int64_t n, float *u_dev, int ckpt_every, float *ckpt_dev, void *stream);

/* Reverse mode of spiir_impulse_forward for a real loss L(u).
 *   grad_u_dev [T][n] complex: dL/dRe u + i dL/dIm u (PyTorch's convention).
 *   ckpt_dev   the checkpoints written by spiir_impulse_forward with the same ckpt_every.
 *   workspace_dev [ceil(n / ckpt_every) + 2][T][F] complex: scratch, overwritten.
 * Outputs [T][F] complex in the same convention:
 *   grad_a1 = sum_k lambda_l[k] conj(y_l[k-1]), grad_b0 = lambda_l[d_l] (0 if d_l >= n),
 *   grad_s0 = conj(a1_l) lambda_l[0], where lambda_l[n] = 0 and
 *   lambda_l[k] = grad_u_t[k] + conj(a1_l) lambda_l[k+1].
 * Parallel over checkpoint segments: each segment's own part of lambda, a double-float scan over the
 * segments for their boundary values, then states recomputed from the checkpoints and the
 * gradients formed segment by segment (added over segments in double-float, in order).  Shared memory
 * grows with ckpt_every: SPIIR_EUNSUPPORTED when it does not fit.  Enqueued on stream. */
int spiir_impulse_backward(int n_templates, int filters_per_template, const float *a1_dev,
                           const float *b0_dev, const int32_t *delay_dev, int64_t n,
                           const float *grad_u_dev, int ckpt_every, const float *ckpt_dev,
                           float *grad_a1_dev, float *grad_b0_dev, float *grad_s0_dev,
                           float *workspace_dev, void *stream);

/* ------------------------------------------------------------------------------------
 * Streaming pipeline: one call per strain chunk runs the whole hot path (filter bank,
 * SNR history of 2 H samples, coherent scan).  Output sample j of a call is geocentric
 * sample (stream position of the chunk start) + j - H: the coherent stage lags the
 * strain by H samples so that every detector's delayed SNR is available.
 * The streaming state (bank states, strain and SNR history, staging buffers) is ordered only
 * by the CUDA stream: every call on one pipeline must use the same stream, and one pipeline
 * must not be driven from two host threads at once.
 * ---------------------------------------------------------------------------------- */

/* bank and sky must have the same n_det and must outlive the pipeline.  max_chunk
 * bounds n in later calls. */
int spiir_pipeline_create(spiir_bank_t bank, spiir_sky_t sky, int64_t max_chunk,
                          spiir_pipeline_t *out);
void spiir_pipeline_destroy(spiir_pipeline_t pipe);
/* Zero all streaming state (bank states, strain and SNR history). */
int spiir_pipeline_reset(spiir_pipeline_t pipe, void *stream);

/* Device buffers: strain_dev [n_det][strain_pitch]; outputs [n_templates][n] as in
 * spiir_coherent_scan; skymap_dev NULL or [n_templates][n_pix][n].  Enqueued on stream. */
int spiir_pipeline_run(spiir_pipeline_t pipe, const float *strain_dev, int64_t strain_pitch,
                       int64_t n, float *max_stat_dev, int32_t *argmax_dev,
                       float *null_stat_dev, float *skymap_dev, void *stream);

/* The whole path from raw strain (Sec. II.A - II.C): strain_dev [n_det][strain_pitch] at the
 * front end's input rate, n_in samples (a positive multiple of its M with n_in / M <= max_chunk),
 * goes through spiir_frontend_run (down-sampling and whitening, its own lags) into a buffer the
 * pipeline owns, then through the step of spiir_pipeline_run with n = n_in / M.  Outputs as for
 * spiir_pipeline_run.  fe must have the bank's n_det; it keeps its own stream of histories, so
 * drive it only through this call while it is attached to a stream of chunks.  Four or more
 * launches on stream.  Errors: SPIIR_EINVAL, SPIIR_ENOMEM (first call), SPIIR_ECUDA. */
int spiir_pipeline_run_frontend(spiir_pipeline_t pipe, spiir_frontend_t fe, const float *strain_dev,
                                int64_t strain_pitch, int64_t n_in, float *max_stat_dev,
                                int32_t *argmax_dev, float *null_stat_dev, float *skymap_dev,
                                void *stream);

/* Same with host buffers: copies the strain [n_det][n] to the device, runs, copies
 * max_stat, argmax and null_stat [n_templates][n] back and synchronises stream.  Host
 * buffers should be page-locked for full copy bandwidth. */
int spiir_pipeline_run_host(spiir_pipeline_t pipe, const float *strain_host, int64_t n,
                            float *max_stat_host, int32_t *argmax_host,
                            float *null_stat_host, void *stream);

/* Asynchronous host-buffer step for streaming: the same work as spiir_pipeline_run_host,
 * enqueued without waiting.  The strain is copied and the chunk processed on stream; the
 * outputs are copied to the host buffers on the pipeline's own copy stream, so that they
 * travel while the next submitted chunk is processed (two device staging sets alternate, and
 * a set is reused only after its copies are done).  strain_host must stay unchanged, and the
 * output buffers must stay valid and unread, until spiir_pipeline_wait returns; page-locked
 * host memory is needed for the copies to overlap.  Chunks are processed in submission order.
 * Errors: SPIIR_EINVAL, SPIIR_ENOMEM (first call: the second staging set), SPIIR_ECUDA. */
int spiir_pipeline_submit_host(spiir_pipeline_t pipe, const float *strain_host, int64_t n,
                               float *max_stat_host, int32_t *argmax_host,
                               float *null_stat_host, void *stream);
/* Block until every submitted step's outputs are in its host buffers. */
int spiir_pipeline_wait(spiir_pipeline_t pipe);
/* The same with a host-side limit: SPIIR_OK once every submitted step is complete, or
 * SPIIR_ETIMEOUT (nothing is cancelled; the steps keep running and a later wait collects them)
 * when timeout_s seconds pass first, so that a caller can detect a stalled stream without
 * blocking.  Errors: SPIIR_EINVAL, SPIIR_ETIMEOUT, SPIIR_ECUDA. */
int spiir_pipeline_wait_for(spiir_pipeline_t pipe, double timeout_s);

/* ------------------------------------------------------------------------------------
 * Batched multirate banks.  Several template banks of uneven size share one strain stream.
 * Every filter runs in one band b at the rate 1 / M_b of the strain (M_b a power of two;
 * M = 1 is the full rate); its delay is in samples of its band.  Per chunk of strain:
 *   x_b[j]  = sum_{i<32} h_b[i] x[j M_b - i]   (Hann-windowed sinc, cutoff 0.8 x the band's
 *             Nyquist, unit DC gain; M = 1 passes x through)
 *   z_b     = the band-b filters of each template on x_b (Eq. (zk), Sec. II.B.1)
 *   z[k]    = sum_b (1 - w) z_b[m-1] + w z_b[m],  m = floor(k / M_b), w = (k mod M_b) / M_b
 *             (one low-rate sample of lag; a band with M = 1 contributes z_b[k], no lag)
 *   coherent scan of z over all templates of all banks (Sec. II.C.1), one H-sample lag as in
 *   the streaming pipeline.
 * The paper filters one rate only (its front end downsamples 16 kHz to 2 kHz by FIR); the
 * band split, the decimation filter and the upsampling rule are this library's definitions.
 * ---------------------------------------------------------------------------------- */

/* templates_per_bank [n_banks]; filter_offsets [T+1] over all templates of all banks in
 * bank order (T = sum of templates_per_bank); a1, b0 [2 F]; delay [F]; band [F] in
 * [0, n_bands); band_factor [n_bands] (powers of two <= 64).  chunk: full-rate samples per
 * call, >= 32 and a multiple of every band factor.  sky must outlive the batch.  All host
 * arrays.  Builds both the per-band banks of the batched path and the per-(bank, band)
 * banks of the plain path. */
int spiir_batch_create(int n_det, int n_banks, const int32_t *templates_per_bank,
                       const int64_t *filter_offsets_host, const float *a1_host,
                       const float *b0_host, const int32_t *delay_host, const int32_t *band_host,
                       int n_bands, const int32_t *band_factor, spiir_sky_t sky, int64_t chunk,
                       spiir_batch_t *out);
void spiir_batch_destroy(spiir_batch_t batch);
int spiir_batch_info(spiir_batch_t batch, int *n_templates, int64_t *n_filters, int *n_work_items);
/* Zero all streaming state of both paths. */
int spiir_batch_reset(spiir_batch_t batch, void *stream);
/* Launch shape of the persistent filter launch (a tuning knob): filters_per_lane,
 * lanes_per_block, steps_per_reduce as in spiir_bank_set_shape; blocks_per_sm 0 = as many as
 * fit.  Keeps the streaming state; drops a captured graph.  Synchronises the device. */
int spiir_batch_set_shape(spiir_batch_t batch, int filters_per_lane, int lanes_per_block,
                          int steps_per_reduce, int blocks_per_sm);
/* Process one chunk.  strain_dev [n_det][chunk] (contiguous); outputs [T][chunk] as in
 * spiir_coherent_scan (templates in bank order).
 *   mode 0: plain path, separate launches per bank and band;
 *   mode 1: batched path, one persistent filter launch, launched eagerly;
 *   mode 2: batched path replayed from a CUDA graph, captured on the first call (and again
 *           whenever the buffer pointers change).
 * A batch streams in one path: switching between mode 0 and modes 1/2 needs
 * spiir_batch_reset (SPIIR_EINVAL otherwise).  Enqueued on stream. */
int spiir_batch_run(spiir_batch_t batch, int mode, const float *strain_dev, float *max_stat_dev,
                    int32_t *argmax_dev, float *null_stat_dev, void *stream);
/* Device time of the persistent filter launch alone (a measurement hook; no counterpart in
 * the paper).  The first call creates two CUDA events and returns *ms = -1; from then on every
 * eager batched chunk (mode 1) records them around its persistent launch, and a call
 * synchronises on the second event and returns the last such launch's time in ms (-1 before
 * one has run).  Graph-replayed chunks are not timed.  Errors: SPIIR_EINVAL, SPIIR_ECUDA. */
int spiir_batch_filter_time(spiir_batch_t batch, float *ms);

#ifdef __cplusplus
}
#endif
#endif /* SPIIR_H */
