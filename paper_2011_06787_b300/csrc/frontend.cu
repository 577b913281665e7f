// Front end (Sec. II.A): the strain of each detector is low-passed and down-sampled from the
// input rate (16384 Hz) by a time-domain FIR filter, then whitened.  The paper whitens in the
// frequency domain, Eq. (whiten): d_w = F^-1[ d~(f) / sqrt(S_n(f)) ]; here the same zero-phase
// response, scaled to unit-variance output, sqrt(2 / (f_s S_n(f))), is applied as a causal
// linear-phase FIR in the time domain, so the front end streams sample by sample with a fixed
// delay instead of collecting segments.
//
//   decimation:  x_2[j] = sum_{i < L_d} h[i] x[j M - i]
//   whitening:   y_I[k] = sum_{i < L_w} w_I[i] x_2,I[k - i]
//
// Device mapping.  k_fe_decimate: one thread per output sample, the block's input window kept
// in shared memory as M phase planes (sample i of the window in plane i mod M, row i / M) so
// that consecutive outputs read consecutive words.  k_fe_whiten: a block computes 128 outputs
// of one detector; a thread owns 8 consecutive outputs and one of 64 slices of the taps, slides
// a 16-register window over the input, and the 64 partial sums of each output are added in a
// fixed order.  Both kernels read the previous segment's samples from a history buffer and
// write the new history to the other buffer of a pair (the next call reads it), so no copy of
// the input is made and blocks never race on the history.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"

struct spiir_frontend_s {
    int n_det = 0, M = 1, Ld = 1, Lw = 1, Lw_pad = 1;
    int64_t max_in = 0;
    float *taps_d = nullptr;      // [Ld] decimation low-pass
    float *taps_w = nullptr;      // [n_det][Lw_pad] whitening, zero beyond Lw
    float *hist16[2] = {nullptr, nullptr};  // [n_det][Ld - 1] input-rate history
    float *hist2[2] = {nullptr, nullptr};   // [n_det][Lw_pad - 1] decimated history
    float *dec = nullptr;         // [n_det][max_in / M] decimated segment
    int par = 0;                  // which history buffer holds the current history
};

namespace spiir {

constexpr int kFeDecOut = 128;          // outputs per block of k_fe_decimate
constexpr int kFeWhOut = 128;           // outputs per block of k_fe_whiten
constexpr int kFeWhQ = 8;               // outputs per thread
constexpr int kFeWhSlices = 64;         // tap slices
constexpr int kFeWhThreads = (kFeWhOut / kFeWhQ) * kFeWhSlices;  // 1024
constexpr int kFeTapAlign = kFeWhSlices * 8;                     // padded tap count granularity
constexpr int kFeMaxLw = 16384 + 1;
constexpr int kFeMaxLd = 8192;
constexpr int kFeMaxM = 64;

// concatenated stream [history (L - 1) | segment (n)]: sample g
__device__ __forceinline__ float cat_at(const float *hist, int L1, const float *seg, int64_t n, int64_t g) {
    if (g < L1) return hist[g];
    const int64_t s = g - L1;
    return s < n ? seg[s] : 0.f;
}

__global__ void __launch_bounds__(kFeDecOut) k_fe_decimate(const float *__restrict__ x, int64_t x_pitch, int64_t n_in,
                                                           const float *__restrict__ hist_in, float *__restrict__ hist_out,
                                                           const float *__restrict__ taps, int Ld, int M,
                                                           float *__restrict__ dec, int64_t dec_pitch) {
    grid_dependents_trigger();  // the whitening grid may be scheduled now
    extern __shared__ float fe_smem[];
    const int det = blockIdx.y;
    const int L1 = Ld - 1;
    const int64_t n_out = n_in / M;
    const float *xr = x + (int64_t)det * x_pitch;
    const float *hr = hist_in + (int64_t)det * L1;
    const int64_t m0 = (int64_t)blockIdx.x * kFeDecOut;
    const int W = (kFeDecOut - 1) * M + Ld;      // window samples of this block
    const int R = (W + M - 1) / M;               // rows per phase plane
    float *h = fe_smem;                          // [Ld]
    float *xs = fe_smem + Ld;                    // [M][R]
    for (int i = threadIdx.x; i < Ld; i += kFeDecOut) h[i] = taps[i];
    for (int i = threadIdx.x; i < M * R; i += kFeDecOut) {
        const int p = i % M, r = i / M;          // window sample r M + p
        xs[p * R + r] = (r * M + p < W) ? cat_at(hr, L1, xr, n_in, m0 * M + r * M + p) : 0.f;
    }
    __syncthreads();
    const int t = threadIdx.x;
    if (m0 + t < n_out) {
        // x_2[m0 + t] = sum_i h[L_d - 1 - i] window[t M + i],  i = q M + p
        float acc = 0.f;
        for (int q = 0, i0 = 0; i0 < Ld; ++q, i0 += M) {
            const int np = min(M, Ld - i0);
            for (int p = 0; p < np; ++p) acc = fmaf(h[Ld - 1 - i0 - p], xs[p * R + t + q], acc);
        }
        dec[(int64_t)det * dec_pitch + m0 + t] = acc;
    }
    if (blockIdx.x == 0) {
        // the new history: the last L_d - 1 samples of [history | segment]
        float *ho = hist_out + (int64_t)det * L1;
        for (int i = threadIdx.x; i < L1; i += kFeDecOut) ho[i] = cat_at(hr, L1, xr, n_in, n_in + i);
    }
}

__global__ void __launch_bounds__(kFeWhThreads) k_fe_whiten(const float *__restrict__ dec, int64_t dec_pitch,
                                                           int64_t n, const float *__restrict__ hist_in,
                                                           float *__restrict__ hist_out, const float *__restrict__ taps,
                                                           int L, float *__restrict__ y, int64_t y_pitch) {
    extern __shared__ float fe_smem[];
    const int det = blockIdx.y;
    const int L1 = L - 1;                        // L is the padded tap count (a multiple of 512)
    const float *dr = dec + (int64_t)det * dec_pitch;
    const float *hr = hist_in + (int64_t)det * L1;
    const int64_t k0 = (int64_t)blockIdx.x * kFeWhOut;
    const int W = kFeWhOut + L1;
    float *w = fe_smem;                          // [L]
    float *xs = fe_smem + L;                     // [W]: concatenated samples k0 .. k0 + W - 1
    float *part = xs + ((W + 3) & ~3);           // [kFeWhSlices][kFeWhOut]
    const float *tw = taps + (int64_t)det * L;
    for (int i = threadIdx.x; i < L; i += kFeWhThreads) w[i] = tw[i];
    // launched as a programmatic dependent of the decimation: its output is complete and
    // visible after this (the taps above do not depend on it)
    grid_dependency_wait();
    for (int i = threadIdx.x; i < W; i += kFeWhThreads) xs[i] = cat_at(hr, L1, dr, n, k0 + i);
    __syncthreads();
    const int og = threadIdx.x % (kFeWhOut / kFeWhQ), sl = threadIdx.x / (kFeWhOut / kFeWhQ);
    const int JT = L / kFeWhSlices;              // taps per slice, a multiple of 8
    const int ja = sl * JT;
    // output og*8 + i needs window sample og*8 + i + L1 - j for tap j
    const int base = og * kFeWhQ + L1;
    float acc[kFeWhQ];
#pragma unroll
    for (int i = 0; i < kFeWhQ; ++i) acc[i] = 0.f;
    // xr[c] = window sample (base - jj - 8 + c), c = 0..15.  xr[0] is first used one step
    // after it is loaded; in the last slice's last step its index can be -1 (clamped, unused).
    float xr[16];
    xr[0] = xs[max(base - ja - 8, 0)];
#pragma unroll
    for (int c = 1; c < 16; ++c) xr[c] = xs[base - ja - 8 + c];
    for (int jj = ja; jj < ja + JT; jj += 8) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const float wj = w[jj + u];
#pragma unroll
            for (int i = 0; i < kFeWhQ; ++i) acc[i] = fmaf(wj, xr[8 - u + i], acc[i]);
        }
        if (jj + 8 < ja + JT) {
#pragma unroll
            for (int c = 15; c >= 8; --c) xr[c] = xr[c - 8];
            xr[0] = xs[max(base - jj - 16, 0)];
#pragma unroll
            for (int c = 1; c < 8; ++c) xr[c] = xs[base - jj - 16 + c];
        }
    }
#pragma unroll
    for (int i = 0; i < kFeWhQ; ++i) part[sl * kFeWhOut + og * kFeWhQ + i] = acc[i];
    __syncthreads();
    for (int o = threadIdx.x; o < kFeWhOut; o += kFeWhThreads) {
        if (k0 + o >= n) continue;
        float s = 0.f;
        for (int q = 0; q < kFeWhSlices; ++q) s += part[q * kFeWhOut + o];
        y[(int64_t)det * y_pitch + k0 + o] = s;
    }
    if (blockIdx.x == 0) {
        float *ho = hist_out + (int64_t)det * L1;
        for (int i = threadIdx.x; i < L1; i += kFeWhThreads) ho[i] = cat_at(hr, L1, dr, n, n + i);
    }
}

static size_t dec_smem(int Ld, int M) {
    const int W = (kFeDecOut - 1) * M + Ld;
    return sizeof(float) * ((size_t)Ld + (size_t)M * ((W + M - 1) / M));
}
static size_t white_smem(int Lpad) {
    const int W = kFeWhOut + Lpad - 1;
    return sizeof(float) * ((size_t)Lpad + (size_t)((W + 3) & ~3) + (size_t)kFeWhSlices * kFeWhOut);
}

}  // namespace spiir

using namespace spiir;

// ---------------------------------------------------------------------------------------
// Host helpers (FP64 design, FP32 taps)

extern "C" int spiir_fir_lowpass(int n_taps, int M, double cutoff, float *taps) {
    clear_error();
    if (n_taps < 1 || n_taps > kFeMaxLd || M < 1 || M > kFeMaxM || !(cutoff > 0.0 && cutoff <= 1.0) || !taps)
        return fail(SPIIR_EINVAL, "n_taps = %d, M = %d, cutoff = %g", n_taps, M, cutoff);
    const double fc = cutoff * 0.5 / M;  // cycles per input sample
    const double c = 0.5 * (n_taps - 1);
    std::vector<double> h(n_taps);
    double sum = 0.0;
    for (int i = 0; i < n_taps; ++i) {
        const double a = 2.0 * fc * (i - c);
        const double sinc = a == 0.0 ? 1.0 : std::sin(M_PI * a) / (M_PI * a);
        const double hann = 0.5 - 0.5 * std::cos(2.0 * M_PI * (i + 0.5) / n_taps);
        h[i] = 2.0 * fc * sinc * hann;
        sum += h[i];
    }
    if (!(std::fabs(sum) > 0.0)) return fail(SPIIR_EINVAL, "the low-pass has zero DC gain");
    for (int i = 0; i < n_taps; ++i) taps[i] = (float)(h[i] / sum);
    return SPIIR_OK;
}

extern "C" int spiir_whitening_kernel(int n_freq, const double *psd, double rate_hz, int n_taps, float *taps) {
    clear_error();
    if (n_freq < 2 || !psd || !taps || !(rate_hz > 0.0))
        return fail(SPIIR_EINVAL, "n_freq = %d, rate_hz = %g", n_freq, rate_hz);
    const int N = 2 * (n_freq - 1);
    if (n_taps < 1 || n_taps % 2 != 1 || n_taps >= N || n_taps > kFeMaxLw)
        return fail(SPIIR_EINVAL, "n_taps = %d must be odd, below 2 (n_freq - 1) = %d and at most %d", n_taps, N,
                    kFeMaxLw);
    std::vector<double> A(n_freq);
    for (int j = 0; j < n_freq; ++j) {
        if (!(psd[j] > 0.0) || !std::isfinite(psd[j])) return fail(SPIIR_EINVAL, "psd[%d] = %g", j, psd[j]);
        A[j] = std::sqrt(2.0 / (rate_hz * psd[j]));
    }
    // a[m] = (1/N) sum_{j=0}^{N-1} A_j e^{2 pi i j m / N} for the real, even A on N points
    const int K = n_taps / 2;
    std::vector<double> cs(N);
    for (int r = 0; r < N; ++r) cs[r] = std::cos(2.0 * M_PI * r / N);
    for (int i = 0; i < n_taps; ++i) {
        const int m = i - K;
        double acc = A[0] + ((m & 1) ? -A[n_freq - 1] : A[n_freq - 1]);
        const int mm = ((m % N) + N) % N;
        for (int j = 1; j < n_freq - 1; ++j) acc += 2.0 * A[j] * cs[(int)(((int64_t)j * mm) % N)];
        const double win = 0.5 - 0.5 * std::cos(2.0 * M_PI * (i + 1) / (n_taps + 1));
        taps[i] = (float)(win * acc / N);
    }
    return SPIIR_OK;
}

// ---------------------------------------------------------------------------------------
// Streaming front end

static void fe_free(spiir_frontend_s *f) {
    if (!f) return;
    dev_free(f->taps_d);
    dev_free(f->taps_w);
    for (int b = 0; b < 2; ++b) {
        dev_free(f->hist16[b]);
        dev_free(f->hist2[b]);
    }
    dev_free(f->dec);
    delete f;
}

extern "C" int spiir_frontend_create(int n_det, int M, int n_dec_taps, const float *dec_taps, int n_white_taps,
                                     const float *white_taps, int64_t max_in, spiir_frontend_t *out) {
    clear_error();
    if (!out) return fail(SPIIR_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_det < 1 || n_det > 65535 || M < 1 || M > kFeMaxM || n_dec_taps < 1 || n_dec_taps > kFeMaxLd ||
        n_white_taps < 1 || n_white_taps > kFeMaxLw || max_in < M || max_in % M != 0)
        return fail(SPIIR_EINVAL, "n_det = %d, M = %d, n_dec_taps = %d, n_white_taps = %d, max_in = %lld", n_det, M,
                    n_dec_taps, n_white_taps, (long long)max_in);
    if (!dec_taps || !white_taps) return fail(SPIIR_EINVAL, "NULL taps");
    for (int i = 0; i < n_dec_taps; ++i)
        if (!std::isfinite(dec_taps[i])) return fail(SPIIR_EINVAL, "dec_taps[%d] is not finite", i);
    for (int64_t i = 0; i < (int64_t)n_det * n_white_taps; ++i)
        if (!std::isfinite(white_taps[i])) return fail(SPIIR_EINVAL, "white_taps[%lld] is not finite", (long long)i);
    spiir_frontend_s *f = new (std::nothrow) spiir_frontend_s();
    if (!f) return fail(SPIIR_ENOMEM, "host allocation of the front end failed");
    f->n_det = n_det;
    f->M = M;
    f->Ld = n_dec_taps;
    f->Lw = n_white_taps;
    f->Lw_pad = (n_white_taps + kFeTapAlign - 1) / kFeTapAlign * kFeTapAlign;
    f->max_in = max_in;
    std::vector<float> wpad((size_t)n_det * f->Lw_pad, 0.f);
    for (int I = 0; I < n_det; ++I)
        std::copy(white_taps + (size_t)I * n_white_taps, white_taps + (size_t)(I + 1) * n_white_taps,
                  wpad.begin() + (size_t)I * f->Lw_pad);
    const size_t h16 = sizeof(float) * (size_t)n_det * std::max(1, n_dec_taps - 1);
    const size_t h2 = sizeof(float) * (size_t)n_det * (f->Lw_pad - 1);
    int rc = dev_alloc((void **)&f->taps_d, sizeof(float) * n_dec_taps, "decimation taps");
    if (rc == SPIIR_OK) rc = dev_alloc((void **)&f->taps_w, sizeof(float) * wpad.size(), "whitening taps");
    for (int b = 0; b < 2 && rc == SPIIR_OK; ++b) {
        rc = dev_alloc((void **)&f->hist16[b], h16, "input history");
        if (rc == SPIIR_OK) rc = dev_alloc((void **)&f->hist2[b], h2, "decimated history");
    }
    if (rc == SPIIR_OK) rc = dev_alloc((void **)&f->dec, sizeof(float) * (size_t)n_det * (max_in / M), "decimated segment");
    if (rc == SPIIR_OK &&
        (cudaMemcpy(f->taps_d, dec_taps, sizeof(float) * n_dec_taps, cudaMemcpyHostToDevice) != cudaSuccess ||
         cudaMemcpy(f->taps_w, wpad.data(), sizeof(float) * wpad.size(), cudaMemcpyHostToDevice) != cudaSuccess))
        rc = fail(SPIIR_ECUDA, "copy of the taps failed");
    for (int b = 0; b < 2 && rc == SPIIR_OK; ++b)
        if (cudaMemset(f->hist16[b], 0, h16) != cudaSuccess || cudaMemset(f->hist2[b], 0, h2) != cudaSuccess)
            rc = fail(SPIIR_ECUDA, "clearing the histories failed");
    if (rc == SPIIR_OK && white_smem(f->Lw_pad) > 48 * 1024 &&
        cudaFuncSetAttribute(k_fe_whiten, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)white_smem(f->Lw_pad)) !=
            cudaSuccess)
        rc = fail(SPIIR_ECUDA, "shared-memory limit of the whitening kernel");
    if (rc == SPIIR_OK && dec_smem(f->Ld, f->M) > 48 * 1024 &&
        cudaFuncSetAttribute(k_fe_decimate, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dec_smem(f->Ld, f->M)) !=
            cudaSuccess)
        rc = fail(SPIIR_ECUDA, "shared-memory limit of the decimation kernel");
    if (rc != SPIIR_OK) {
        fe_free(f);
        return rc;
    }
    *out = f;
    return SPIIR_OK;
}

extern "C" void spiir_frontend_destroy(spiir_frontend_t f) { fe_free(f); }

extern "C" int spiir_frontend_info(spiir_frontend_t f, int *n_det, int *M, int64_t *max_in) {
    if (!f) return fail(SPIIR_EINVAL, "front end is NULL");
    if (n_det) *n_det = f->n_det;
    if (M) *M = f->M;
    if (max_in) *max_in = f->max_in;
    return SPIIR_OK;
}

extern "C" int spiir_frontend_reset(spiir_frontend_t f, void *stream) {
    clear_error();
    if (!f) return fail(SPIIR_EINVAL, "front end is NULL");
    const size_t h16 = sizeof(float) * (size_t)f->n_det * std::max(1, f->Ld - 1);
    const size_t h2 = sizeof(float) * (size_t)f->n_det * (f->Lw_pad - 1);
    for (int b = 0; b < 2; ++b) {
        SPIIR_CUDA_TRY(cudaMemsetAsync(f->hist16[b], 0, h16, (cudaStream_t)stream));
        SPIIR_CUDA_TRY(cudaMemsetAsync(f->hist2[b], 0, h2, (cudaStream_t)stream));
    }
    f->par = 0;
    return SPIIR_OK;
}

extern "C" int spiir_frontend_run(spiir_frontend_t f, const float *strain, int64_t strain_pitch, int64_t n_in,
                                  float *out, int64_t out_pitch, void *stream) {
    clear_error();
    if (!f) return fail(SPIIR_EINVAL, "front end is NULL");
    if (!strain || !out) return fail(SPIIR_EINVAL, "NULL buffer");
    if (n_in < f->M || n_in % f->M != 0 || n_in > f->max_in)
        return fail(SPIIR_EINVAL, "n_in = %lld must be a positive multiple of %d and at most %lld", (long long)n_in,
                    f->M, (long long)f->max_in);
    const int64_t n_out = n_in / f->M;
    if (strain_pitch < n_in || out_pitch < n_out)
        return fail(SPIIR_EINVAL, "strain_pitch %lld < n_in or out_pitch %lld < n_in / M", (long long)strain_pitch,
                    (long long)out_pitch);
    cudaStream_t s = (cudaStream_t)stream;
    const int p = f->par;
    const int64_t dec_pitch = f->max_in / f->M;
    k_fe_decimate<<<dim3((unsigned)((n_out + kFeDecOut - 1) / kFeDecOut), (unsigned)f->n_det), kFeDecOut,
                    dec_smem(f->Ld, f->M), s>>>(strain, strain_pitch, n_in, f->hist16[p], f->hist16[1 - p], f->taps_d,
                                                f->Ld, f->M, f->dec, dec_pitch);
    SPIIR_CUDA_TRY(cudaGetLastError());
    // programmatic dependent launch: the whitening blocks stage their taps while the decimation
    // drains
    SPIIR_CUDA_TRY(launch_dependent(k_fe_whiten, dim3((unsigned)((n_out + kFeWhOut - 1) / kFeWhOut), (unsigned)f->n_det),
                                    dim3(kFeWhThreads), white_smem(f->Lw_pad), s, (const float *)f->dec, dec_pitch,
                                    n_out, (const float *)f->hist2[p], f->hist2[1 - p], (const float *)f->taps_w,
                                    f->Lw_pad, out, out_pitch));
    f->par = 1 - p;
    return SPIIR_OK;
}
