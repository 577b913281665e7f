// Batched multirate filter banks with one persistent filter launch per chunk, captured in a
// CUDA graph, and the per-bank launch path it is compared with.
//
// A batch holds several template banks of uneven size.  Every filter belongs to a band b
// with decimation factor M_b (the full-rate band has M = 1).  Per strain chunk:
//   1. each detector's strain is low-pass filtered (32-tap Hann-windowed sinc, cutoff 0.8 x
//      the band's Nyquist, unit DC gain) and decimated: x_b[j] = sum_i h_b[i] x[j M_b - i];
//   2. the filters of band b run on x_b (Sec. II.B.1, Eq. (zk));
//   3. each band's SNR is upsampled linearly to the full rate,
//      z[k] = (1 - w) z_b[m - 1] + w z_b[m],  m = floor(k / M_b),  w = (k mod M_b) / M_b,
//      and the bands are summed per template and detector;
//   4. the coherent scan runs over all templates of all banks (Sec. II.C.1).
// Batched path: the filters of all banks are regrouped into one bank per band, and one
// persistent launch covers every (band, template block, detector) work item, largest first,
// taken from a shared counter.  The whole chunk -- copies, decimation, persistent filter
// launch, upsampling, coherent scan and history updates -- is captured once into a CUDA graph
// and replayed per chunk.  Plain path: one bank per (bank, band) with its own launches, one
// upsampling and one coherent launch per bank.
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cstdio>
#include <cmath>
#include <numeric>
#include <vector>

#include "bank.cuh"
#include "coherent.cuh"

namespace spiir {

constexpr int kFirTaps = 32;

struct UpArgs {
    const float2 *zb[kMaxBands];  // band SNR rows [rows][n_det][pitch]; entry 0 = previous chunk's last sample
    int64_t pitch[kMaxBands];
    const int *rowmap[kMaxBands];  // [nT] row of each template in zb[b], -1 when it has no band-b filters
    int M[kMaxBands];
    int n_bands;
    int nT;                        // templates handled by this launch
    int n_det;
    int64_t n;                     // full-rate samples
    float2 *z;                     // [nT][n_det][zpitch], written at zoff + k
    int64_t zpitch, zoff;
    int rows[kMaxBands];           // rows of each zb (bounds-checked debug build)
    int *status;
};

__global__ void k_upsample_sum(const __grid_constant__ UpArgs a) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= a.n) return;
    const int t = blockIdx.y / a.n_det, det = blockIdx.y % a.n_det;
    float2 acc = make_float2(0.f, 0.f);
    for (int b = 0; b < a.n_bands; ++b) {
        const int row = a.rowmap[b][t];
        if (row < 0) continue;
#ifdef SPIIR_CHECKED
        if (row >= a.rows[b]) {
            report_bounds(a.status, 20 + b);
            continue;
        }
#endif
        const float2 *r = a.zb[b] + ((int64_t)row * a.n_det + det) * a.pitch[b];
        const int M = a.M[b];
        float2 v;
        if (M == 1) {
            v = r[1 + k];
        } else {
            const int64_t m = k / M;
            const float w = (float)(k - m * M) / (float)M;
            const float2 lo = r[m], hi = r[m + 1];
            v = make_float2(fmaf(w, hi.x, (1.f - w) * lo.x), fmaf(w, hi.y, (1.f - w) * lo.y));
        }
        acc.x += v.x;
        acc.y += v.y;
    }
    a.z[((int64_t)t * a.n_det + det) * a.zpitch + a.zoff + k] = acc;
}

// x_b[j] = sum_i h[i] x[j M - i]; xin rows hold kFirTaps - 1 history samples, then the chunk.
__global__ void k_decimate(const float *xin, int64_t xin_pitch, const float *taps, int M, int64_t nb, float *out,
                           int64_t out_pitch) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int det = blockIdx.y;
    if (j >= nb) return;
    const float *x = xin + det * xin_pitch + (kFirTaps - 1) + j * M;
    float acc = 0.f;
#pragma unroll
    for (int i = 0; i < kFirTaps; ++i) acc = fmaf(taps[i], x[-i], acc);
    out[det * out_pitch + j] = acc;
}

// FP64 design of the decimation low-pass, rounded to FP32.
static void fir_design(int M, float *h) {
    if (M == 1) {
        for (int i = 0; i < kFirTaps; ++i) h[i] = i == 0 ? 1.f : 0.f;
        return;
    }
    const double pi = 3.14159265358979323846;
    const double fc = 0.8 * 0.5 / M, c = 0.5 * (kFirTaps - 1);
    double v[kFirTaps], sum = 0;
    for (int i = 0; i < kFirTaps; ++i) {
        const double x = 2.0 * fc * (i - c);
        const double sinc = (x == 0.0) ? 1.0 : std::sin(pi * x) / (pi * x);
        const double win = 0.5 - 0.5 * std::cos(2.0 * pi * (i + 0.5) / kFirTaps);
        v[i] = 2.0 * fc * sinc * win;
        sum += v[i];
    }
    for (int i = 0; i < kFirTaps; ++i) h[i] = (float)(v[i] / sum);
}

}  // namespace spiir

using namespace spiir;

struct spiir_batch_s {
    int n_det = 0, n_banks = 0, n_bands = 0;
    int M[kMaxBands] = {1, 1, 1, 1};
    int64_t chunk = 0;
    int T = 0;
    int64_t F = 0;
    std::vector<int> bank_t0;  // [n_banks + 1]
    spiir_sky_s *sky = nullptr;
    int H = 0;
    // batched: one bank per band over all templates with filters in that band
    spiir_bank_s *band_bank[kMaxBands] = {nullptr, nullptr, nullptr, nullptr};
    float2 *zb[kMaxBands] = {nullptr, nullptr, nullptr, nullptr};
    int zb_rows[kMaxBands] = {0, 0, 0, 0};
    int *rowmap[kMaxBands] = {nullptr, nullptr, nullptr, nullptr};  // [T]
    int4 *items = nullptr;
    int n_items = 0;
    int *counter = nullptr;
    int shape_S = 8, shape_NL = 128, shape_R = 32, blocks_per_sm = 0;
    // plain: one bank per (bank, band)
    std::vector<spiir_bank_s *> pbank;          // [n_banks * n_bands]
    std::vector<float2 *> pzb;                  // [n_banks * n_bands]
    std::vector<int *> prowmap;                 // [n_banks * n_bands], rows over the bank's templates
    // shared buffers
    float *xin = nullptr;       // [n_det][xin_pitch]: FIR history, then the chunk
    int64_t xin_pitch = 0;
    float *xdec[kMaxBands] = {nullptr, nullptr, nullptr, nullptr};  // [n_det][chunk / M]
    float *taps = nullptr;      // [n_bands][32]
    float2 *zpad = nullptr;     // [T][n_det][zpitch]: 2 H history, then the chunk
    float2 *ztmp = nullptr;
    int64_t zpitch = 0;
    int last_mode = -1;
    // graph of the batched chunk
    cudaGraphExec_t gexec = nullptr;
    cudaStream_t cap = nullptr;
    const float *g_strain = nullptr;
    float *g_ms = nullptr, *g_nl = nullptr;
    int32_t *g_am = nullptr;
    // CUDA events around the persistent filter launch of eager batched chunks (mode 1)
    cudaEvent_t f_ev[2] = {nullptr, nullptr};
    bool f_timed = false;
};

namespace spiir {

static int64_t band_len(const spiir_batch_s *B, int b) { return B->chunk / B->M[b]; }
static int64_t zb_pitch(const spiir_batch_s *B, int b) { return band_len(B, b) + 1; }

static void batch_free(spiir_batch_s *B) {
    if (!B) return;
    if (B->gexec) cudaGraphExecDestroy(B->gexec);
    if (B->cap) cudaStreamDestroy(B->cap);
    for (int i = 0; i < 2; ++i)
        if (B->f_ev[i]) cudaEventDestroy(B->f_ev[i]);
    for (int b = 0; b < kMaxBands; ++b) {
        if (B->band_bank[b]) spiir_bank_destroy(B->band_bank[b]);
        dev_free(B->zb[b]);
        dev_free(B->rowmap[b]);
        dev_free(B->xdec[b]);
    }
    for (auto *p : B->pbank)
        if (p) spiir_bank_destroy(p);
    for (auto *p : B->pzb) dev_free(p);
    for (auto *p : B->prowmap) dev_free(p);
    dev_free(B->items);
    dev_free(B->counter);
    dev_free(B->xin);
    dev_free(B->taps);
    dev_free(B->zpad);
    dev_free(B->ztmp);
    delete B;
}

// A bank made of the band-b filters of templates [t_lo, t_hi); rows lists the templates that
// have at least one such filter (the bank's templates, in order).
static int make_band_bank(spiir_batch_s *B, const int64_t *off, const float *a1, const float *b0, const int32_t *delay,
                          const int32_t *band, int b, int t_lo, int t_hi, spiir_bank_s **out, std::vector<int> &rows) {
    std::vector<int64_t> o{0};
    std::vector<float> A, Bv;
    std::vector<int32_t> D;
    rows.clear();
    for (int t = t_lo; t < t_hi; ++t) {
        int64_t cnt = 0;
        for (int64_t l = off[t]; l < off[t + 1]; ++l) {
            if (band[l] != b) continue;
            A.push_back(a1[2 * l]);
            A.push_back(a1[2 * l + 1]);
            Bv.push_back(b0[2 * l]);
            Bv.push_back(b0[2 * l + 1]);
            D.push_back(delay[l]);
            ++cnt;
        }
        if (cnt > 0) {
            rows.push_back(t);
            o.push_back(o.back() + cnt);
        }
    }
    *out = nullptr;
    if (rows.empty()) return SPIIR_OK;
    SPIIR_TRY(spiir_bank_create(B->n_det, (int)rows.size(), o.data(), A.data(), Bv.data(), D.data(), out));
    return bank_prepare(*out, band_len(B, b), 0);
}

static int upload_rowmap(const std::vector<int> &rows, int t_lo, int nT, int **dst) {
    std::vector<int> m(nT, -1);
    for (size_t r = 0; r < rows.size(); ++r) m[rows[r] - t_lo] = (int)r;
    SPIIR_TRY(dev_alloc((void **)dst, sizeof(int) * nT, "band row map"));
    SPIIR_CUDA_TRY(cudaMemcpy(*dst, m.data(), sizeof(int) * nT, cudaMemcpyHostToDevice));
    return SPIIR_OK;
}

// Work items of the persistent launch, largest first: (band, block, detector).
static int build_items(spiir_batch_s *B) {
    struct It {
        int64_t cost;
        int4 v;
    };
    std::vector<It> its;
    for (int b = 0; b < B->n_bands; ++b) {
        spiir_bank_s *k = B->band_bank[b];
        if (!k) continue;
        for (int c = 0; c < k->n_cta; ++c)
            for (int d = 0; d < B->n_det; ++d)
                its.push_back({(int64_t)k->h_active[c] * band_len(B, b), make_int4(b, c, d, 0)});
    }
    std::stable_sort(its.begin(), its.end(), [](const It &x, const It &y) { return x.cost > y.cost; });
    std::vector<int4> v(its.size());
    for (size_t i = 0; i < its.size(); ++i) v[i] = its[i].v;
    dev_free(B->items);
    B->items = nullptr;
    B->n_items = (int)v.size();
    SPIIR_TRY(dev_alloc((void **)&B->items, sizeof(int4) * std::max<size_t>(1, v.size()), "work items"));
    if (!v.empty()) SPIIR_CUDA_TRY(cudaMemcpy(B->items, v.data(), sizeof(int4) * v.size(), cudaMemcpyHostToDevice));
    return SPIIR_OK;
}

// strain -> FIR history buffer; decimated bands -> xdec
static int stage_and_decimate(spiir_batch_s *B, const float *strain, cudaStream_t s) {
    const int L = kFirTaps - 1;
    SPIIR_CUDA_TRY(cudaMemcpy2DAsync(B->xin + L, B->xin_pitch * 4, strain, B->chunk * 4, B->chunk * 4, B->n_det,
                                     cudaMemcpyDeviceToDevice, s));
    for (int b = 0; b < B->n_bands; ++b) {
        if (B->M[b] == 1) continue;
        const int64_t nb = band_len(B, b);
        k_decimate<<<dim3((unsigned)((nb + 127) / 128), B->n_det), 128, 0, s>>>(B->xin, B->xin_pitch, B->taps + b * kFirTaps,
                                                                             B->M[b], nb, B->xdec[b], nb);
        SPIIR_CUDA_TRY(cudaGetLastError());
    }
    // the last L samples become the FIR history (chunk >= 32, so the ranges do not overlap)
    SPIIR_CUDA_TRY(cudaMemcpy2DAsync(B->xin, B->xin_pitch * 4, B->xin + B->chunk, B->xin_pitch * 4, L * 4, B->n_det,
                                     cudaMemcpyDeviceToDevice, s));
    return SPIIR_OK;
}

static const float *band_input(spiir_batch_s *B, int b, const float *strain) {
    return B->M[b] == 1 ? strain : B->xdec[b];
}

static int zpad_history(spiir_batch_s *B, cudaStream_t s) {
    if (B->H == 0) return SPIIR_OK;
    const size_t w = 2 * B->H * sizeof(float2), pitch = B->zpitch * sizeof(float2), rows = (size_t)B->T * B->n_det;
    if (B->chunk >= 2 * B->H) {
        SPIIR_CUDA_TRY(cudaMemcpy2DAsync(B->zpad, pitch, B->zpad + B->chunk, pitch, w, rows, cudaMemcpyDeviceToDevice, s));
    } else {
        SPIIR_CUDA_TRY(cudaMemcpy2DAsync(B->ztmp, w, B->zpad + B->chunk, pitch, w, rows, cudaMemcpyDeviceToDevice, s));
        SPIIR_CUDA_TRY(cudaMemcpy2DAsync(B->zpad, pitch, B->ztmp, w, w, rows, cudaMemcpyDeviceToDevice, s));
    }
    return SPIIR_OK;
}

static int band_history(float2 *zb, int rows, int n_det, int64_t nb, int64_t pitch, cudaStream_t s) {
    // the last band sample of every row becomes entry 0 of that row
    SPIIR_CUDA_TRY(cudaMemcpy2DAsync(zb, pitch * sizeof(float2), zb + nb, pitch * sizeof(float2), sizeof(float2),
                                     (size_t)rows * n_det, cudaMemcpyDeviceToDevice, s));
    return SPIIR_OK;
}

static int run_upsample(spiir_batch_s *B, float2 *const *zb, const int *const *rowmap, int t0, int nT,
                        cudaStream_t s) {
    UpArgs u{};
    for (int b = 0; b < B->n_bands; ++b) {
        u.zb[b] = zb[b];
        u.pitch[b] = zb_pitch(B, b);
        u.rowmap[b] = rowmap[b];
        u.M[b] = B->M[b];
    }
    u.n_bands = B->n_bands;
    u.nT = nT;
    u.n_det = B->n_det;
    u.n = B->chunk;
    u.z = B->zpad + (int64_t)t0 * B->n_det * B->zpitch;
    u.zpitch = B->zpitch;
    u.zoff = 2 * B->H;
    u.status = device_status_word();
    for (int b = 0; b < B->n_bands; ++b) u.rows[b] = (t0 == 0 && nT == B->T) ? B->zb_rows[b] : 1 << 30;
    const unsigned rows = (unsigned)nT * B->n_det;
    k_upsample_sum<<<dim3((unsigned)((B->chunk + 255) / 256), rows), 256, 0, s>>>(u);
    SPIIR_CUDA_TRY(cudaGetLastError());
    return SPIIR_OK;
}

#ifdef SPIIR_CHECKED
#define SPIIR_DEBUG_SYNC(what)                                                                   \
    do {                                                                                         \
        cudaStreamCaptureStatus cs_ = cudaStreamCaptureStatusNone;                               \
        cudaStreamIsCapturing(s, &cs_);                                                          \
        if (cs_ == cudaStreamCaptureStatusNone) {                                                \
            const cudaError_t e_ = cudaStreamSynchronize(s);                                     \
            int st_ = 0;                                                                         \
            cudaMemcpy(&st_, device_status_word(), sizeof(int), cudaMemcpyDeviceToHost);         \
            fprintf(stderr, "[checked] %s: %s status=0x%x\n", what, cudaGetErrorString(e_), st_); \
        }                                                                                        \
    } while (0)
#else
#define SPIIR_DEBUG_SYNC(what) \
    do {                       \
    } while (0)
#endif

// Bands without filters anywhere still need a valid (all -1) row map; their zb is unused.
static int batched_chunk(spiir_batch_s *B, const float *strain, float *ms, int32_t *am, float *nl, cudaStream_t s) {
    SPIIR_TRY(stage_and_decimate(B, strain, s));
    SPIIR_DEBUG_SYNC("decimate");
    PersistArgs p{};
    size_t smem = 0;
    for (int b = 0; b < B->n_bands; ++b) {
        spiir_bank_s *k = B->band_bank[b];
        if (!k) continue;
        const int64_t nb = band_len(B, b);
        // band input -> the bank's strain window (its history stays in place)
        SPIIR_CUDA_TRY(cudaMemcpy2DAsync(k->xbuf[k->cur] + k->D_pad, k->xpitch * 4, band_input(B, b, strain),
                                         (B->M[b] == 1 ? B->chunk : nb) * 4, nb * 4, B->n_det,
                                         cudaMemcpyDeviceToDevice, s));
        p.banks[b] = bank_args(k, B->zb[b] + 1, zb_pitch(B, b), nb);
        p.banks[b].z_elems = zb_pitch(B, b) * B->zb_rows[b] * B->n_det - 1;
        smem = std::max(smem, bank_smem_bytes(k));
    }
    p.items = B->items;
    p.n_items = B->n_items;
    p.counter = B->counter;
    SPIIR_CUDA_TRY(cudaMemsetAsync(B->counter, 0, sizeof(int), s));
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    SPIIR_CUDA_TRY(cudaStreamIsCapturing(s, &cs));
    const bool timed = cs == cudaStreamCaptureStatusNone && B->f_ev[0] && B->f_ev[1];
    if (timed) SPIIR_CUDA_TRY(cudaEventRecord(B->f_ev[0], s));
    if (B->n_items > 0) SPIIR_TRY(bank_launch_persistent(p, B->shape_S, B->shape_NL, B->shape_R, B->blocks_per_sm, smem, s));
    if (timed) {
        SPIIR_CUDA_TRY(cudaEventRecord(B->f_ev[1], s));
        B->f_timed = true;
    }
    SPIIR_DEBUG_SYNC("persistent filter");
    // bands with long delays: add the later delay pieces of their split templates
    for (int b = 0; b < B->n_bands; ++b)
        if (B->band_bank[b]) SPIIR_TRY(bank_piece_sum(B->band_bank[b], B->zb[b] + 1, zb_pitch(B, b), band_len(B, b), s));
    for (int b = 0; b < B->n_bands; ++b) {
        spiir_bank_s *k = B->band_bank[b];
        if (!k || k->D_pad == 0) continue;
        // move the last D_pad samples to the front through the bank's second window buffer
        float *x = k->xbuf[k->cur], *tmp = k->xbuf[1 - k->cur];
        const int64_t nb = band_len(B, b);
        SPIIR_CUDA_TRY(cudaMemcpy2DAsync(tmp, k->xpitch * 4, x + nb, k->xpitch * 4, k->D_pad * 4, B->n_det,
                                         cudaMemcpyDeviceToDevice, s));
        SPIIR_CUDA_TRY(cudaMemcpy2DAsync(x, k->xpitch * 4, tmp, k->xpitch * 4, k->D_pad * 4, B->n_det,
                                         cudaMemcpyDeviceToDevice, s));
    }
    SPIIR_DEBUG_SYNC("history moves");
    SPIIR_TRY(run_upsample(B, B->zb, B->rowmap, 0, B->T, s));
    SPIIR_DEBUG_SYNC("upsample");
    for (int b = 0; b < B->n_bands; ++b)
        if (B->band_bank[b]) SPIIR_TRY(band_history(B->zb[b], B->zb_rows[b], B->n_det, band_len(B, b), zb_pitch(B, b), s));
    SPIIR_DEBUG_SYNC("band history");
    SPIIR_TRY(coherent_scan(B->sky, B->zpad, B->zpitch, B->T, B->chunk, ms, am, nl, nullptr, s));
    SPIIR_DEBUG_SYNC("coherent");
    const int rz = zpad_history(B, s);
    SPIIR_DEBUG_SYNC("zpad history");
    return rz;
}

static int plain_chunk(spiir_batch_s *B, const float *strain, float *ms, int32_t *am, float *nl, cudaStream_t s) {
    SPIIR_TRY(stage_and_decimate(B, strain, s));
    for (int k = 0; k < B->n_banks; ++k) {
        const int t0 = B->bank_t0[k], nT = B->bank_t0[k + 1] - t0;
        float2 *zb[kMaxBands] = {nullptr, nullptr, nullptr, nullptr};
        const int *rm[kMaxBands] = {nullptr, nullptr, nullptr, nullptr};
        for (int b = 0; b < B->n_bands; ++b) {
            const int i = k * B->n_bands + b;
            zb[b] = B->pzb[i];
            rm[b] = B->prowmap[i];
            spiir_bank_s *pb = B->pbank[i];
            if (!pb) continue;
            const int64_t nb = band_len(B, b);
            SPIIR_TRY(bank_filter(pb, band_input(B, b, strain), B->M[b] == 1 ? B->chunk : nb, nb, B->pzb[i] + 1,
                                  zb_pitch(B, b), s));
        }
        SPIIR_TRY(run_upsample(B, zb, rm, t0, nT, s));
        for (int b = 0; b < B->n_bands; ++b) {
            const int i = k * B->n_bands + b;
            if (B->pbank[i]) SPIIR_TRY(band_history(B->pzb[i], B->pbank[i]->T, B->n_det, band_len(B, b), zb_pitch(B, b), s));
        }
        SPIIR_TRY(coherent_scan(B->sky, B->zpad + (int64_t)t0 * B->n_det * B->zpitch, B->zpitch, nT, B->chunk,
                                ms + (int64_t)t0 * B->chunk, am + (int64_t)t0 * B->chunk, nl + (int64_t)t0 * B->chunk,
                                nullptr, s));
    }
    return zpad_history(B, s);
}

static int batch_zero_state(spiir_batch_s *B, cudaStream_t s) {
    SPIIR_CUDA_TRY(cudaMemsetAsync(B->xin, 0, sizeof(float) * B->xin_pitch * B->n_det, s));
    SPIIR_CUDA_TRY(cudaMemsetAsync(B->zpad, 0, sizeof(float2) * B->zpitch * B->T * B->n_det, s));
    for (int b = 0; b < B->n_bands; ++b) {
        if (B->band_bank[b]) {
            SPIIR_TRY(spiir_bank_reset(B->band_bank[b], s));
            SPIIR_CUDA_TRY(cudaMemsetAsync(B->zb[b], 0, sizeof(float2) * zb_pitch(B, b) * B->zb_rows[b] * B->n_det, s));
        }
    }
    for (size_t i = 0; i < B->pbank.size(); ++i) {
        if (!B->pbank[i]) continue;
        SPIIR_TRY(spiir_bank_reset(B->pbank[i], s));
        const int b = (int)(i % B->n_bands);
        SPIIR_CUDA_TRY(cudaMemsetAsync(B->pzb[i], 0, sizeof(float2) * zb_pitch(B, b) * B->pbank[i]->T * B->n_det, s));
    }
    return SPIIR_OK;
}

}  // namespace spiir

extern "C" int spiir_batch_create(int n_det, int n_banks, const int32_t *tpb, const int64_t *off, const float *a1,
                                  const float *b0, const int32_t *delay, const int32_t *band, int n_bands,
                                  const int32_t *band_factor, spiir_sky_t sky, int64_t chunk, spiir_batch_t *out) {
    clear_error();
    if (!out) return fail(SPIIR_EINVAL, "out is NULL");
    *out = nullptr;
    if (!tpb || !off || !band || !band_factor) return fail(SPIIR_EINVAL, "NULL argument");
    if (n_banks < 1 || n_det < 1) return fail(SPIIR_EINVAL, "bad n_banks or n_det");
    if (n_bands < 1 || n_bands > kMaxBands) return fail(SPIIR_EINVAL, "n_bands = %d outside [1, %d]", n_bands, kMaxBands);
    int Mmax = 1;
    for (int b = 0; b < n_bands; ++b) {
        const int M = band_factor[b];
        if (M < 1 || M > 64 || (M & (M - 1))) return fail(SPIIR_EINVAL, "band factor %d must be a power of two <= 64", M);
        Mmax = std::max(Mmax, M);
    }
    if (chunk < 32 || chunk % Mmax != 0 || chunk > (1 << 20))
        return fail(SPIIR_EINVAL, "chunk %lld must be >= 32 and a multiple of every band factor", (long long)chunk);
    int T = 0;
    for (int k = 0; k < n_banks; ++k) {
        if (tpb[k] < 1) return fail(SPIIR_EINVAL, "bank %d has no templates", k);
        T += tpb[k];
    }
    if (off[0] != 0) return fail(SPIIR_EINVAL, "filter_offsets[0] must be 0");
    for (int t = 0; t < T; ++t)
        if (off[t + 1] < off[t]) return fail(SPIIR_EINVAL, "filter_offsets decrease at template %d", t);
    const int64_t F = off[T];
    for (int64_t l = 0; l < F; ++l)
        if (band[l] < 0 || band[l] >= n_bands) return fail(SPIIR_EINVAL, "filter %lld has band %d", (long long)l, band[l]);
    if (!sky) return fail(SPIIR_EINVAL, "sky is NULL");
    if (sky->n_det != n_det) return fail(SPIIR_EINVAL, "sky has %d detectors, the batch %d", sky->n_det, n_det);
    spiir_batch_s *B = new (std::nothrow) spiir_batch_s();
    if (!B) return fail(SPIIR_ENOMEM, "host allocation of the batch failed");
    B->n_det = n_det;
    B->n_banks = n_banks;
    B->n_bands = n_bands;
    for (int b = 0; b < n_bands; ++b) B->M[b] = band_factor[b];
    B->chunk = chunk;
    B->T = T;
    B->F = F;
    B->sky = sky;
    B->H = sky->halo;
    B->bank_t0.assign(n_banks + 1, 0);
    for (int k = 0; k < n_banks; ++k) B->bank_t0[k + 1] = B->bank_t0[k] + tpb[k];
    int rc = SPIIR_OK;
    std::vector<int> rows;
    // batched: one bank per band
    for (int b = 0; b < n_bands && rc == SPIIR_OK; ++b) {
        rc = make_band_bank(B, off, a1, b0, delay, band, b, 0, T, &B->band_bank[b], rows);
        if (rc == SPIIR_OK) rc = upload_rowmap(rows, 0, T, &B->rowmap[b]);
        B->zb_rows[b] = (int)rows.size();
        if (rc == SPIIR_OK && !rows.empty())
            rc = dev_alloc((void **)&B->zb[b], sizeof(float2) * zb_pitch(B, b) * rows.size() * n_det, "band SNR");
    }
    // plain: one bank per (bank, band)
    B->pbank.assign((size_t)n_banks * n_bands, nullptr);
    B->pzb.assign((size_t)n_banks * n_bands, nullptr);
    B->prowmap.assign((size_t)n_banks * n_bands, nullptr);
    for (int k = 0; k < n_banks && rc == SPIIR_OK; ++k)
        for (int b = 0; b < n_bands && rc == SPIIR_OK; ++b) {
            const int i = k * n_bands + b, t0 = B->bank_t0[k], t1 = B->bank_t0[k + 1];
            rc = make_band_bank(B, off, a1, b0, delay, band, b, t0, t1, &B->pbank[i], rows);
            if (rc == SPIIR_OK) rc = upload_rowmap(rows, t0, t1 - t0, &B->prowmap[i]);
            if (rc == SPIIR_OK && !rows.empty())
                rc = dev_alloc((void **)&B->pzb[i], sizeof(float2) * zb_pitch(B, b) * rows.size() * n_det, "band SNR");
        }
    B->xin_pitch = ((kFirTaps - 1 + chunk + 3) / 4) * 4;
    if (rc == SPIIR_OK) rc = dev_alloc((void **)&B->xin, sizeof(float) * B->xin_pitch * n_det, "FIR history");
    for (int b = 0; b < n_bands && rc == SPIIR_OK; ++b)
        if (B->M[b] > 1) rc = dev_alloc((void **)&B->xdec[b], sizeof(float) * band_len(B, b) * n_det, "band strain");
    std::vector<float> taps((size_t)n_bands * kFirTaps);
    for (int b = 0; b < n_bands; ++b) fir_design(B->M[b], taps.data() + b * kFirTaps);
    if (rc == SPIIR_OK) rc = dev_alloc((void **)&B->taps, sizeof(float) * taps.size(), "FIR taps");
    if (rc == SPIIR_OK && cudaMemcpy(B->taps, taps.data(), sizeof(float) * taps.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        rc = fail(SPIIR_ECUDA, "copy of FIR taps failed");
    B->zpitch = ((2 * B->H + chunk + 1) / 2) * 2;
    if (rc == SPIIR_OK) rc = dev_alloc((void **)&B->zpad, sizeof(float2) * B->zpitch * T * n_det, "SNR rows");
    if (rc == SPIIR_OK && B->H > 0)
        rc = dev_alloc((void **)&B->ztmp, sizeof(float2) * 2 * B->H * T * n_det, "SNR history scratch");
    if (rc == SPIIR_OK) rc = dev_alloc((void **)&B->counter, sizeof(int), "work counter");
    // one launch shape for every band bank (the persistent kernel is compiled per shape)
    if (rc == SPIIR_OK) {
        int64_t fmax = 0;
        for (int b = 0; b < n_bands; ++b) {
            spiir_bank_s *k = B->band_bank[b];
            if (!k) continue;
            for (int t = 0; t < k->T; ++t) fmax = std::max(fmax, k->offsets[t + 1] - k->offsets[t]);
        }
        B->shape_S = 8;
        B->shape_NL = fmax > 1024 ? 256 : 128;
        if (fmax > 2048) B->shape_S = 16;
        for (int b = 0; b < n_bands && rc == SPIIR_OK; ++b)
            if (B->band_bank[b])
                rc = spiir_bank_set_shape(B->band_bank[b], B->shape_S, B->shape_NL, B->shape_R, B->band_bank[b]->c_tile);
    }
    if (rc == SPIIR_OK) rc = build_items(B);
    if (rc == SPIIR_OK && !device_status_word()) rc = fail(SPIIR_ECUDA, "device status word unavailable");
    if (rc == SPIIR_OK) rc = batch_zero_state(B, 0);
    if (rc == SPIIR_OK && cudaDeviceSynchronize() != cudaSuccess) rc = fail(SPIIR_ECUDA, "initialisation failed");
    if (rc != SPIIR_OK) {
        batch_free(B);
        return rc;
    }
    *out = B;
    return SPIIR_OK;
}

extern "C" void spiir_batch_destroy(spiir_batch_t B) { batch_free(B); }

extern "C" int spiir_batch_info(spiir_batch_t B, int *n_templates, int64_t *n_filters, int *n_items) {
    if (!B) return fail(SPIIR_EINVAL, "batch is NULL");
    if (n_templates) *n_templates = B->T;
    if (n_filters) *n_filters = B->F;
    if (n_items) *n_items = B->n_items;
    return SPIIR_OK;
}

extern "C" int spiir_batch_reset(spiir_batch_t B, void *stream) {
    if (!B) return fail(SPIIR_EINVAL, "batch is NULL");
    SPIIR_TRY(batch_zero_state(B, (cudaStream_t)stream));
    B->last_mode = -1;
    return SPIIR_OK;
}

extern "C" int spiir_batch_set_shape(spiir_batch_t B, int filters_per_lane, int lanes_per_block, int steps_per_reduce,
                                     int blocks_per_sm) {
    clear_error();
    if (!B) return fail(SPIIR_EINVAL, "batch is NULL");
    if (blocks_per_sm < 0 || blocks_per_sm > 8) return fail(SPIIR_EINVAL, "blocks_per_sm must be in [0, 8]");
    for (int b = 0; b < B->n_bands; ++b) {
        spiir_bank_s *k = B->band_bank[b];
        if (!k) continue;
        int oS, oNL, oR, oT;
        spiir_bank_get_shape(k, &oS, &oNL, &oR, &oT);
        const int rc = spiir_bank_set_shape(k, filters_per_lane, lanes_per_block, steps_per_reduce, oT);
        if (rc != SPIIR_OK) {
            char msg[512];
            spiir_last_error(msg, sizeof msg);
            // put back the banks already changed; their device arrays moved, so the work
            // list is rebuilt and a captured graph dropped
            for (int c = 0; c < b; ++c)
                if (B->band_bank[c]) spiir_bank_set_shape(B->band_bank[c], B->shape_S, B->shape_NL, B->shape_R, oT);
            if (b > 0) {
                build_items(B);
                if (B->gexec) {
                    cudaGraphExecDestroy(B->gexec);
                    B->gexec = nullptr;
                }
            }
            return fail(rc, "%s", msg);
        }
    }
    B->shape_S = filters_per_lane;
    B->shape_NL = lanes_per_block;
    B->shape_R = steps_per_reduce;
    B->blocks_per_sm = blocks_per_sm;
    SPIIR_TRY(build_items(B));
    if (B->gexec) {
        cudaGraphExecDestroy(B->gexec);
        B->gexec = nullptr;
    }
    return SPIIR_OK;
}

extern "C" int spiir_batch_filter_time(spiir_batch_t B, float *ms) {
    clear_error();
    if (!B || !ms) return fail(SPIIR_EINVAL, "NULL argument");
    if (!B->f_ev[0]) {
        for (int i = 0; i < 2; ++i) SPIIR_CUDA_TRY(cudaEventCreate(&B->f_ev[i]));
        *ms = -1.f;
        return SPIIR_OK;
    }
    if (!B->f_timed) {
        *ms = -1.f;
        return SPIIR_OK;
    }
    SPIIR_CUDA_TRY(cudaEventSynchronize(B->f_ev[1]));
    SPIIR_CUDA_TRY(cudaEventElapsedTime(ms, B->f_ev[0], B->f_ev[1]));
    return SPIIR_OK;
}

extern "C" int spiir_batch_run(spiir_batch_t B, int mode, const float *strain, float *ms, int32_t *am, float *nl,
                               void *stream) {
    clear_error();
    // host-side range per chunk for profilers (a no-op without one)
    struct Range {
        Range() { nvtxRangePushA("spiir.batch_chunk"); }
        ~Range() { nvtxRangePop(); }
    } range;
    if (!B) return fail(SPIIR_EINVAL, "batch is NULL");
    if (!strain || !ms || !am || !nl) return fail(SPIIR_EINVAL, "NULL buffer");
    if (mode < 0 || mode > 2) return fail(SPIIR_EINVAL, "mode %d not in {0, 1, 2}", mode);
    const bool batched_state = mode != 0;
    if (B->last_mode >= 0 && (B->last_mode != 0) != batched_state)
        return fail(SPIIR_EINVAL, "the batch streamed in another mode; call spiir_batch_reset first");
    cudaStream_t s = (cudaStream_t)stream;
    int rc;
    if (mode == 0) {
        rc = plain_chunk(B, strain, ms, am, nl, s);
    } else if (mode == 1) {
        rc = batched_chunk(B, strain, ms, am, nl, s);
    } else {
        if (B->gexec && (B->g_strain != strain || B->g_ms != ms || B->g_am != am || B->g_nl != nl)) {
            cudaGraphExecDestroy(B->gexec);
            B->gexec = nullptr;
        }
        if (!B->gexec) {
            if (!B->cap) SPIIR_CUDA_TRY(cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking));
            cudaGraph_t g = nullptr;
            SPIIR_CUDA_TRY(cudaStreamBeginCapture(B->cap, cudaStreamCaptureModeThreadLocal));
            const int crc = batched_chunk(B, strain, ms, am, nl, B->cap);
            const cudaError_t ce = cudaStreamEndCapture(B->cap, &g);
            if (crc != SPIIR_OK) {
                if (g) cudaGraphDestroy(g);
                return crc;
            }
            if (ce != cudaSuccess) return fail(SPIIR_ECUDA, "graph capture failed: %s", cudaGetErrorString(ce));
            const cudaError_t ie = cudaGraphInstantiate(&B->gexec, g, 0);
            cudaGraphDestroy(g);
            if (ie != cudaSuccess) return fail(SPIIR_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(ie));
            B->g_strain = strain;
            B->g_ms = ms;
            B->g_am = am;
            B->g_nl = nl;
        }
        const cudaError_t le = cudaGraphLaunch(B->gexec, s);
        rc = le == cudaSuccess ? SPIIR_OK : fail(SPIIR_ECUDA, "graph launch failed: %s", cudaGetErrorString(le));
    }
    if (rc == SPIIR_OK) B->last_mode = mode;
    return rc;
}
