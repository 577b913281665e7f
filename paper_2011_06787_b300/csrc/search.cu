// Candidate-driven streaming search (Sec. II.C.1 - II.C.3): one call per strain chunk runs
//   1. the filter bank (Sec. II.B.1, Eq. (zk)) into a ring of SNR history,
//   2. single-detector candidate selection over one span of the stream (the largest |z| over
//      the bank per sample, over the threshold, one per template per second),
//   3. the coherent statistic at every candidate at zero lag on the foreground sky,
//   4. the time-shift background: shifts 1 .. n_shifts on the background sky,
//   5. xi_C^2 (Sec. II.C.2) at every candidate for zero lag and every shift.
// Nothing returns to the host: the candidate count stays on the device and the later stages
// read it there.
//
// SNR ring.  Each (template, detector) row holds 2 L entries; stream sample s lives at
// s mod L and again at s mod L + L, so that any L consecutive stream samples are contiguous
// in the row and the candidate kernels read them with a plain (pitch, offset) view.  The
// filter bank writes a chunk at p = s mod L (p + n <= 2 L), and two copies mirror the part
// below L up by L and the part above L down by L.
//
// Span.  The span analysed by a call ends La = 2 H + Nj samples before the last filtered
// sample (H the larger sky halo, Nj the xi^2 half-width), the most the zero-lag stages read
// past a candidate; the background and xi^2 read back at most
// Hb = n_shifts (n_det - 1) step + 2 H + Nj samples before it.  L = Hb + chunk + La.
//
// Overlapped mode.  A call forks an internal stream from the caller's, runs the candidate
// stages there on the span the ring surrounded before the call, while the filter bank writes
// the new chunk on the caller's stream, and joins back.  The ring then keeps one chunk more,
// L = Hb + 2 chunk + La, so that the chunk being written (samples pos .. pos + chunk - 1, at
// the ring positions of samples pos - L ..) never shares an entry with the span's reads
// (samples pos - L + chunk .. pos - 1).
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>

#include "bank.cuh"
#include "coherent.cuh"

struct spiir_search_s {
    spiir_bank_s *bank = nullptr;
    spiir_sky_s *fg = nullptr, *bg = nullptr;
    int n_det = 0, T = 0, n_lags = 0, per_second = 0, n_shifts = 0, step = 0, max_cand = 0;
    float threshold = 0.f;
    int64_t chunk = 0;
    int64_t hist = 0, look = 0, L = 0;  // Hb, La, ring length
    int64_t pos = 0;                    // stream samples filtered so far
    float2 *ring = nullptr;             // [T][n_det][2 L]
    float2 *A = nullptr;                // [T][2 n_lags + 1]
    void *ws = nullptr;
    size_t ws_bytes = 0;
    bool overlap = false;
    cudaStream_t side = nullptr;          // overlapped mode: the candidate stages' stream
    cudaEvent_t fork = nullptr, join = nullptr;
};

namespace spiir {

static void search_free(spiir_search_s *s) {
    if (!s) return;
    dev_free(s->ring);
    dev_free(s->A);
    dev_free(s->ws);
    if (s->side) cudaStreamDestroy(s->side);
    if (s->fork) cudaEventDestroy(s->fork);
    if (s->join) cudaEventDestroy(s->join);
    delete s;
}

static int64_t floor_mod(int64_t a, int64_t m) {
    const int64_t r = a % m;
    return r < 0 ? r + m : r;
}

}  // namespace spiir

using namespace spiir;

extern "C" int spiir_search_create(spiir_bank_t bank, spiir_sky_t sky_fg, spiir_sky_t sky_bg, const float *A_dev,
                                   int n_lags, int64_t chunk, float threshold, int per_second, int n_shifts,
                                   int shift_step, int max_cand, int flags, spiir_search_t *out) {
    clear_error();
    if (!out) return fail(SPIIR_EINVAL, "out is NULL");
    *out = nullptr;
    if (!bank || !sky_fg || !sky_bg || !A_dev) return fail(SPIIR_EINVAL, "NULL argument");
    if (sky_fg->n_det != bank->n_det || sky_bg->n_det != bank->n_det)
        return fail(SPIIR_EINVAL, "the skies have %d and %d detectors, the bank %d", sky_fg->n_det, sky_bg->n_det,
                    bank->n_det);
    if (bank->n_det < 2) return fail(SPIIR_EINVAL, "a coherent search needs at least 2 detectors");
    if (n_lags < 0 || n_lags > 1024) return fail(SPIIR_EINVAL, "n_lags = %d outside [0, 1024]", n_lags);
    if (chunk < 1 || chunk > (1 << 24)) return fail(SPIIR_EINVAL, "chunk = %lld outside [1, 2^24]", (long long)chunk);
    if (per_second < 1) return fail(SPIIR_EINVAL, "per_second = %d < 1", per_second);
    if (!(threshold >= 0.f) || !std::isfinite(threshold)) return fail(SPIIR_EINVAL, "threshold must be finite and >= 0");
    if (n_shifts < 0 || shift_step < 0) return fail(SPIIR_EINVAL, "n_shifts = %d, shift_step = %d", n_shifts, shift_step);
    if (max_cand < 1 || (int64_t)max_cand * std::max(n_shifts, 1) > INT32_MAX)
        return fail(SPIIR_EINVAL, "max_cand = %d (with %d shifts)", max_cand, n_shifts);
    if (((uintptr_t)A_dev) % 8) return fail(SPIIR_EINVAL, "A_dev must be 8-byte aligned");
    if (flags & ~SPIIR_SEARCH_OVERLAP) return fail(SPIIR_EINVAL, "unknown flags 0x%x", flags);
    spiir_search_s *s = new (std::nothrow) spiir_search_s();
    if (!s) return fail(SPIIR_ENOMEM, "host allocation of the search failed");
    s->bank = bank;
    s->fg = sky_fg;
    s->bg = sky_bg;
    s->n_det = bank->n_det;
    s->T = bank->T;
    s->n_lags = n_lags;
    s->per_second = per_second;
    s->n_shifts = n_shifts;
    s->step = shift_step;
    s->max_cand = max_cand;
    s->threshold = threshold;
    s->chunk = chunk;
    const int64_t H = std::max(sky_fg->halo, sky_bg->halo);
    s->look = 2 * H + n_lags;
    s->hist = (int64_t)n_shifts * (s->n_det - 1) * shift_step + 2 * H + n_lags;
    s->overlap = (flags & SPIIR_SEARCH_OVERLAP) != 0;
    s->L = s->hist + (s->overlap ? 2 : 1) * chunk + s->look;
    const size_t ring_bytes = sizeof(float2) * (size_t)s->T * s->n_det * 2 * (size_t)s->L;
    int rc = dev_alloc((void **)&s->ring, ring_bytes, "SNR ring");
    if (rc == SPIIR_OK && s->overlap &&
        (cudaStreamCreateWithFlags(&s->side, cudaStreamNonBlocking) != cudaSuccess ||
         cudaEventCreateWithFlags(&s->fork, cudaEventDisableTiming) != cudaSuccess ||
         cudaEventCreateWithFlags(&s->join, cudaEventDisableTiming) != cudaSuccess))
        rc = fail(SPIIR_ECUDA, "stream or event creation failed");
    if (rc == SPIIR_OK) rc = dev_alloc((void **)&s->A, sizeof(float2) * (size_t)s->T * (2 * n_lags + 1), "autocorrelations");
    if (rc == SPIIR_OK) rc = spiir_select_workspace_bytes(s->T, s->n_det, chunk, per_second, &s->ws_bytes);
    if (rc == SPIIR_OK) rc = dev_alloc(&s->ws, s->ws_bytes, "selection workspace");
    if (rc == SPIIR_OK && cudaMemset(s->ring, 0, ring_bytes) != cudaSuccess) rc = fail(SPIIR_ECUDA, "cudaMemset failed");
    if (rc == SPIIR_OK && cudaMemset(s->ws, 0, s->ws_bytes) != cudaSuccess) rc = fail(SPIIR_ECUDA, "cudaMemset failed");
    if (rc == SPIIR_OK &&
        cudaMemcpy(s->A, A_dev, sizeof(float2) * (size_t)s->T * (2 * n_lags + 1), cudaMemcpyDeviceToDevice) != cudaSuccess)
        rc = fail(SPIIR_ECUDA, "copy of the autocorrelations failed");
    if (rc == SPIIR_OK) rc = bank_prepare(bank, chunk, 0);
    if (rc == SPIIR_OK && cudaDeviceSynchronize() != cudaSuccess) rc = fail(SPIIR_ECUDA, "initialisation failed");
    if (rc != SPIIR_OK) {
        search_free(s);
        return rc;
    }
    *out = s;
    return SPIIR_OK;
}

extern "C" void spiir_search_destroy(spiir_search_t s) { search_free(s); }

extern "C" int spiir_search_info(spiir_search_t s, int64_t *ring_len, int64_t *history, int64_t *lag,
                                 int64_t *next_span_start) {
    if (!s) return fail(SPIIR_EINVAL, "search is NULL");
    if (ring_len) *ring_len = s->L;
    if (history) *history = s->hist;
    if (lag) *lag = s->look;
    if (next_span_start) *next_span_start = s->pos - (s->overlap ? s->chunk : 0) - s->look;
    return SPIIR_OK;
}

extern "C" int spiir_search_reset(spiir_search_t s, void *stream) {
    if (!s) return fail(SPIIR_EINVAL, "search is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    SPIIR_TRY(spiir_bank_reset(s->bank, stream));
    SPIIR_CUDA_TRY(cudaMemsetAsync(s->ring, 0, sizeof(float2) * (size_t)s->T * s->n_det * 2 * (size_t)s->L, st));
    s->pos = 0;
    return SPIIR_OK;
}

namespace spiir {

// The chunk's SNR into the ring at p = pos mod L, then its mirror image.
static int filter_into_ring(spiir_search_s *s, const float *strain_dev, int64_t strain_pitch, cudaStream_t st) {
    const int64_t n = s->chunk, L = s->L, P2 = 2 * L;
    const size_t rows = (size_t)s->T * s->n_det, pitch_b = sizeof(float2) * (size_t)P2;
    const int64_t p = floor_mod(s->pos, L);
    SPIIR_TRY(bank_filter(s->bank, strain_dev, strain_pitch, n, s->ring + p, P2, st));
    if (p < L) {
        const int64_t w = std::min(p + n, L) - p;
        if (cudaMemcpy2DAsync(s->ring + p + L, pitch_b, s->ring + p, pitch_b, sizeof(float2) * w, rows,
                              cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return fail(SPIIR_ECUDA, "mirror copy failed");
    }
    if (p + n > L) {
        const int64_t w = p + n - L;
        if (cudaMemcpy2DAsync(s->ring, pitch_b, s->ring + L, pitch_b, sizeof(float2) * w, rows,
                              cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return fail(SPIIR_ECUDA, "mirror copy failed");
    }
    return SPIIR_OK;
}

// The candidate stages on the span [S0, S0 + n): entry off + k of a row is stream sample
// S0 + k, and the entries off - Hb .. off + n + La are the consecutive samples they read.
static int candidate_stages(spiir_search_s *s, int64_t S0, int32_t *cand_dev, int32_t *n_cand_dev,
                            float *fg_max_dev, int32_t *fg_argmax_dev, float *fg_null_dev, float *fg_xi2_dev,
                            float *bg_max_dev, int32_t *bg_argmax_dev, float *bg_null_dev, float *bg_xi2_dev,
                            cudaStream_t st) {
    const int64_t n = s->chunk, L = s->L, P2 = 2 * L;
    const int64_t off = floor_mod(S0 - s->hist, L) + s->hist;
    const float *ring = reinterpret_cast<const float *>(s->ring);
    void *stream = (void *)st;
    // 2. selection
    SPIIR_TRY(spiir_select_candidates(s->T, s->n_det, ring, P2, off, n, s->threshold, s->per_second, s->ws,
                                      s->ws_bytes, cand_dev, s->max_cand, n_cand_dev, stream));
    // 3. zero lag on the foreground sky; 4. shifts 1 .. n_shifts on the background sky
    SPIIR_TRY(spiir_coherent_candidates(s->fg, s->T, ring, P2, off, cand_dev, n_cand_dev, s->max_cand, 0, 1, s->step,
                                        fg_max_dev, fg_argmax_dev, fg_null_dev, stream));
    if (s->n_shifts > 0)
        SPIIR_TRY(spiir_coherent_candidates(s->bg, s->T, ring, P2, off, cand_dev, n_cand_dev, s->max_cand, 1,
                                            s->n_shifts, s->step, bg_max_dev, bg_argmax_dev, bg_null_dev, stream));
    // 5. xi_C^2 at each candidate's coherent argmax, zero lag and every shift
    const float *A = reinterpret_cast<const float *>(s->A);
    SPIIR_TRY(spiir_xi2_candidates(s->fg, s->T, ring, P2, off, A, s->n_lags, cand_dev, n_cand_dev, s->max_cand, 0, 1,
                                   s->step, fg_argmax_dev, fg_xi2_dev, nullptr, stream));
    if (s->n_shifts > 0)
        SPIIR_TRY(spiir_xi2_candidates(s->bg, s->T, ring, P2, off, A, s->n_lags, cand_dev, n_cand_dev, s->max_cand,
                                       1, s->n_shifts, s->step, bg_argmax_dev, bg_xi2_dev, nullptr, stream));
    return SPIIR_OK;
}

}  // namespace spiir

extern "C" int spiir_search_run(spiir_search_t s, const float *strain_dev, int64_t strain_pitch, int32_t *cand_dev,
                                int32_t *n_cand_dev, float *fg_max_dev, int32_t *fg_argmax_dev, float *fg_null_dev,
                                float *fg_xi2_dev, float *bg_max_dev, int32_t *bg_argmax_dev, float *bg_null_dev,
                                float *bg_xi2_dev, int64_t *span_start, void *stream) {
    clear_error();
    if (!s) return fail(SPIIR_EINVAL, "search is NULL");
    if (!strain_dev || strain_pitch < s->chunk) return fail(SPIIR_EINVAL, "strain is NULL or its pitch below the chunk");
    if (!cand_dev || !n_cand_dev || !fg_max_dev || !fg_argmax_dev || !fg_null_dev || !fg_xi2_dev)
        return fail(SPIIR_EINVAL, "NULL output pointer");
    if (s->n_shifts > 0 && (!bg_max_dev || !bg_argmax_dev || !bg_null_dev || !bg_xi2_dev))
        return fail(SPIIR_EINVAL, "NULL background output pointer");
    if (((uintptr_t)cand_dev) % 16) return fail(SPIIR_EINVAL, "cand_dev must be 16-byte aligned");
    cudaStream_t st = (cudaStream_t)stream;
    nvtxRangePushA("spiir.search_chunk");
    const int64_t n = s->chunk;
    int rc = SPIIR_OK;
    int64_t S0 = 0;
    if (!s->overlap) {
        // 1. the chunk into the ring, then the span that the ring now surrounds
        rc = filter_into_ring(s, strain_dev, strain_pitch, st);
        if (rc == SPIIR_OK) {
            s->pos += n;
            S0 = s->pos - n - s->look;
            rc = candidate_stages(s, S0, cand_dev, n_cand_dev, fg_max_dev, fg_argmax_dev, fg_null_dev, fg_xi2_dev,
                                  bg_max_dev, bg_argmax_dev, bg_null_dev, bg_xi2_dev, st);
        }
    } else {
        // the span the ring surrounded before this call, on the internal stream, beside the
        // filter bank's new chunk on the caller's stream; then the caller's stream waits
        S0 = s->pos - n - s->look;
        if (cudaEventRecord(s->fork, st) != cudaSuccess || cudaStreamWaitEvent(s->side, s->fork, 0) != cudaSuccess) {
            nvtxRangePop();
            return fail(SPIIR_ECUDA, "stream fork failed");
        }
        rc = candidate_stages(s, S0, cand_dev, n_cand_dev, fg_max_dev, fg_argmax_dev, fg_null_dev, fg_xi2_dev,
                              bg_max_dev, bg_argmax_dev, bg_null_dev, bg_xi2_dev, s->side);
        const int rc_f = rc == SPIIR_OK ? filter_into_ring(s, strain_dev, strain_pitch, st) : rc;
        // joined whatever happened, so that the caller's stream never runs ahead of the stages
        const bool joined = cudaEventRecord(s->join, s->side) == cudaSuccess &&
                            cudaStreamWaitEvent(st, s->join, 0) == cudaSuccess;
        rc = rc_f;
        if (rc == SPIIR_OK && !joined) rc = fail(SPIIR_ECUDA, "stream join failed");
        if (rc == SPIIR_OK) s->pos += n;
    }
    nvtxRangePop();
    if (rc == SPIIR_OK && span_start) *span_start = S0;
    return rc;
}
