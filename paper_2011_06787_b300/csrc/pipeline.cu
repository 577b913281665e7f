// Streaming pipeline: per strain chunk, filter bank -> SNR rows with 2 H samples of
// history -> coherent scan.  Output sample j of a call is geocentric sample
// (chunk start) + j - H, so that the SNR of every detector at k + Delta_I(p) is
// available when the scan runs.
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <chrono>
#include <thread>

#include "bank.cuh"
#include "coherent.cuh"

struct spiir_pipeline_s {
    spiir_bank_s *bank = nullptr;
    spiir_sky_s *sky = nullptr;
    int64_t max_chunk = 0;
    int H = 0;
    int64_t pitch = 0;  // float2 entries per SNR row: 2 H history + max_chunk
    float2 *zpad[2] = {nullptr, nullptr};
    int cur = 0;
    // device staging for the host-buffer entry point
    float *strain_dev = nullptr;
    float *ms_dev = nullptr, *nl_dev = nullptr;
    int32_t *am_dev = nullptr;
    float *fe_out = nullptr;  // [n_det][max_chunk]: front-end output of spiir_pipeline_run_frontend
    // asynchronous host-buffer steps: two staging sets alternate; the outputs of a step go to
    // the host on the copy stream while the next step runs (set 0 is the staging above)
    bool async_ready = false;
    cudaStream_t copy = nullptr;
    cudaEvent_t computed[2] = {nullptr, nullptr}, copied[2] = {nullptr, nullptr};
    float *strain2[2] = {nullptr, nullptr}, *ms2[2] = {nullptr, nullptr}, *nl2[2] = {nullptr, nullptr};
    int32_t *am2[2] = {nullptr, nullptr};
    int abuf = 0;
};

namespace spiir {

static void pipe_free(spiir_pipeline_s *p) {
    if (!p) return;
    if (p->copy) {
        cudaStreamSynchronize(p->copy);
        cudaStreamDestroy(p->copy);
    }
    for (int b = 0; b < 2; ++b) {
        if (p->computed[b]) cudaEventDestroy(p->computed[b]);
        if (p->copied[b]) cudaEventDestroy(p->copied[b]);
    }
    dev_free(p->strain2[1]);
    dev_free(p->ms2[1]);
    dev_free(p->nl2[1]);
    dev_free(p->am2[1]);
    dev_free(p->zpad[0]);
    dev_free(p->zpad[1]);
    dev_free(p->strain_dev);
    dev_free(p->ms_dev);
    dev_free(p->nl_dev);
    dev_free(p->am_dev);
    dev_free(p->fe_out);
    delete p;
}

// Host-side NVTX range (a no-op unless a profiler is attached), closed at scope exit.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

static int pipe_run(spiir_pipeline_s *p, const float *strain, int64_t spitch, int64_t n, float *ms, int32_t *am,
                    float *nl, float *map, cudaStream_t s) {
    NvtxRange chunk("spiir.chunk");
    const int T = p->bank->T, nd = p->bank->n_det, H = p->H;
    float2 *z = p->zpad[p->cur];
    {
        NvtxRange r("spiir.filter_bank");
        SPIIR_TRY(bank_filter(p->bank, strain, spitch, n, z + 2 * H, p->pitch, s));
    }
    {
        NvtxRange r("spiir.coherent_scan");
        SPIIR_TRY(coherent_scan(p->sky, z, p->pitch, T, n, ms, am, nl, map, s));
    }
    const int nxt = 1 - p->cur;
    if (H > 0)
        SPIIR_CUDA_TRY(cudaMemcpy2DAsync(p->zpad[nxt], p->pitch * sizeof(float2), z + n, p->pitch * sizeof(float2),
                                         2 * H * sizeof(float2), (size_t)T * nd, cudaMemcpyDeviceToDevice, s));
    p->cur = nxt;
    return SPIIR_OK;
}

// Lazily created resources of the asynchronous host-buffer steps.
static int async_init(spiir_pipeline_s *p) {
    if (p->async_ready) return SPIIR_OK;
    // each resource is created once; a call that failed part-way resumes where it stopped
    const int T = p->bank->T, nd = p->bank->n_det;
    const int64_t m = p->max_chunk;
    if (!p->copy) SPIIR_CUDA_TRY(cudaStreamCreateWithFlags(&p->copy, cudaStreamNonBlocking));
    for (int b = 0; b < 2; ++b) {
        if (!p->computed[b]) SPIIR_CUDA_TRY(cudaEventCreateWithFlags(&p->computed[b], cudaEventDisableTiming));
        if (!p->copied[b]) SPIIR_CUDA_TRY(cudaEventCreateWithFlags(&p->copied[b], cudaEventDisableTiming));
    }
    p->strain2[0] = p->strain_dev;
    p->ms2[0] = p->ms_dev;
    p->nl2[0] = p->nl_dev;
    p->am2[0] = p->am_dev;
    if (!p->strain2[1]) SPIIR_TRY(dev_alloc((void **)&p->strain2[1], sizeof(float) * nd * m, "strain staging"));
    if (!p->ms2[1]) SPIIR_TRY(dev_alloc((void **)&p->ms2[1], sizeof(float) * T * m, "max staging"));
    if (!p->nl2[1]) SPIIR_TRY(dev_alloc((void **)&p->nl2[1], sizeof(float) * T * m, "null staging"));
    if (!p->am2[1]) SPIIR_TRY(dev_alloc((void **)&p->am2[1], sizeof(int32_t) * T * m, "argmax staging"));
    p->async_ready = true;
    return SPIIR_OK;
}

}  // namespace spiir

using namespace spiir;

extern "C" int spiir_pipeline_create(spiir_bank_t bank, spiir_sky_t sky, int64_t max_chunk, spiir_pipeline_t *out) {
    clear_error();
    if (!out) return fail(SPIIR_EINVAL, "out is NULL");
    *out = nullptr;
    if (!bank || !sky) return fail(SPIIR_EINVAL, "bank or sky is NULL");
    if (bank->n_det != sky->n_det)
        return fail(SPIIR_EINVAL, "bank has %d detectors, sky tables %d", bank->n_det, sky->n_det);
    if (max_chunk < 1 || max_chunk > (1 << 24)) return fail(SPIIR_EINVAL, "max_chunk = %lld", (long long)max_chunk);
    spiir_pipeline_s *p = new (std::nothrow) spiir_pipeline_s();
    if (!p) return fail(SPIIR_ENOMEM, "host allocation of the pipeline failed");
    p->bank = bank;
    p->sky = sky;
    p->max_chunk = max_chunk;
    p->H = sky->halo;
    p->pitch = ((2 * p->H + max_chunk + 1) / 2) * 2;
    const size_t zbytes = sizeof(float2) * (size_t)p->pitch * bank->T * bank->n_det;
    int rc = SPIIR_OK;
    for (int i = 0; i < 2 && rc == SPIIR_OK; ++i) {
        rc = dev_alloc((void **)&p->zpad[i], zbytes, "SNR rows");
        if (rc == SPIIR_OK && cudaMemset(p->zpad[i], 0, zbytes) != cudaSuccess) rc = fail(SPIIR_ECUDA, "memset failed");
    }
    if (rc == SPIIR_OK) rc = dev_alloc((void **)&p->strain_dev, sizeof(float) * bank->n_det * max_chunk, "strain staging");
    if (rc == SPIIR_OK) rc = dev_alloc((void **)&p->ms_dev, sizeof(float) * bank->T * max_chunk, "max staging");
    if (rc == SPIIR_OK) rc = dev_alloc((void **)&p->nl_dev, sizeof(float) * bank->T * max_chunk, "null staging");
    if (rc == SPIIR_OK) rc = dev_alloc((void **)&p->am_dev, sizeof(int32_t) * bank->T * max_chunk, "argmax staging");
    if (rc != SPIIR_OK) {
        pipe_free(p);
        return rc;
    }
    *out = p;
    return SPIIR_OK;
}

extern "C" void spiir_pipeline_destroy(spiir_pipeline_t p) { pipe_free(p); }

extern "C" int spiir_pipeline_reset(spiir_pipeline_t p, void *stream) {
    if (!p) return fail(SPIIR_EINVAL, "pipeline is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    SPIIR_TRY(spiir_bank_reset(p->bank, stream));
    const size_t zbytes = sizeof(float2) * (size_t)p->pitch * p->bank->T * p->bank->n_det;
    for (int i = 0; i < 2; ++i) SPIIR_CUDA_TRY(cudaMemsetAsync(p->zpad[i], 0, zbytes, s));
    return SPIIR_OK;
}

extern "C" int spiir_pipeline_run(spiir_pipeline_t p, const float *strain, int64_t spitch, int64_t n, float *ms,
                                  int32_t *am, float *nl, float *map, void *stream) {
    clear_error();
    if (!p) return fail(SPIIR_EINVAL, "pipeline is NULL");
    if (!strain || !ms || !am || !nl) return fail(SPIIR_EINVAL, "NULL buffer");
    if (n < 1 || n > p->max_chunk) return fail(SPIIR_EINVAL, "n = %lld outside [1, %lld]", (long long)n, (long long)p->max_chunk);
    if (spitch < n) return fail(SPIIR_EINVAL, "strain_pitch < n");
    return pipe_run(p, strain, spitch, n, ms, am, nl, map, (cudaStream_t)stream);
}

extern "C" int spiir_pipeline_run_frontend(spiir_pipeline_t p, spiir_frontend_t fe, const float *strain_dev,
                                           int64_t strain_pitch, int64_t n_in, float *ms, int32_t *am, float *nl,
                                           float *map, void *stream) {
    clear_error();
    if (!p || !fe) return fail(SPIIR_EINVAL, "pipeline or front end is NULL");
    if (!strain_dev || !ms || !am || !nl) return fail(SPIIR_EINVAL, "NULL buffer");
    int nd = 0, M = 1;
    int64_t max_in = 0;
    SPIIR_TRY(spiir_frontend_info(fe, &nd, &M, &max_in));
    if (nd != p->bank->n_det) return fail(SPIIR_EINVAL, "front end has %d detectors, the bank %d", nd, p->bank->n_det);
    if (n_in < M || n_in % M != 0 || n_in / M > p->max_chunk)
        return fail(SPIIR_EINVAL, "n_in = %lld must be a positive multiple of %d with n_in / %d <= %lld",
                    (long long)n_in, M, M, (long long)p->max_chunk);
    if (!p->fe_out)
        SPIIR_TRY(dev_alloc((void **)&p->fe_out, sizeof(float) * (size_t)nd * p->max_chunk, "front-end output"));
    cudaStream_t s = (cudaStream_t)stream;
    NvtxRange r("spiir.frontend_chunk");
    SPIIR_TRY(spiir_frontend_run(fe, strain_dev, strain_pitch, n_in, p->fe_out, p->max_chunk, stream));
    return pipe_run(p, p->fe_out, p->max_chunk, n_in / M, ms, am, nl, map, s);
}

extern "C" int spiir_pipeline_run_host(spiir_pipeline_t p, const float *strain_host, int64_t n, float *ms_host,
                                       int32_t *am_host, float *nl_host, void *stream) {
    clear_error();
    if (!p) return fail(SPIIR_EINVAL, "pipeline is NULL");
    if (!strain_host || !ms_host || !am_host || !nl_host) return fail(SPIIR_EINVAL, "NULL buffer");
    if (n < 1 || n > p->max_chunk) return fail(SPIIR_EINVAL, "n = %lld outside [1, %lld]", (long long)n, (long long)p->max_chunk);
    cudaStream_t s = (cudaStream_t)stream;
    const int T = p->bank->T, nd = p->bank->n_det;
    if (p->async_ready) SPIIR_CUDA_TRY(cudaStreamSynchronize(p->copy));  // staging set 0 is free
    SPIIR_CUDA_TRY(cudaMemcpyAsync(p->strain_dev, strain_host, sizeof(float) * nd * n, cudaMemcpyHostToDevice, s));
    SPIIR_TRY(pipe_run(p, p->strain_dev, n, n, p->ms_dev, p->am_dev, p->nl_dev, nullptr, s));
    SPIIR_CUDA_TRY(cudaMemcpyAsync(ms_host, p->ms_dev, sizeof(float) * T * n, cudaMemcpyDeviceToHost, s));
    SPIIR_CUDA_TRY(cudaMemcpyAsync(am_host, p->am_dev, sizeof(int32_t) * T * n, cudaMemcpyDeviceToHost, s));
    SPIIR_CUDA_TRY(cudaMemcpyAsync(nl_host, p->nl_dev, sizeof(float) * T * n, cudaMemcpyDeviceToHost, s));
    SPIIR_CUDA_TRY(cudaStreamSynchronize(s));
    return SPIIR_OK;
}

extern "C" int spiir_pipeline_submit_host(spiir_pipeline_t p, const float *strain_host, int64_t n, float *ms_host,
                                          int32_t *am_host, float *nl_host, void *stream) {
    clear_error();
    if (!p) return fail(SPIIR_EINVAL, "pipeline is NULL");
    if (!strain_host || !ms_host || !am_host || !nl_host) return fail(SPIIR_EINVAL, "NULL buffer");
    if (n < 1 || n > p->max_chunk) return fail(SPIIR_EINVAL, "n = %lld outside [1, %lld]", (long long)n, (long long)p->max_chunk);
    SPIIR_TRY(async_init(p));
    cudaStream_t s = (cudaStream_t)stream;
    const int T = p->bank->T, nd = p->bank->n_det;
    const int b = p->abuf;
    // the staging set's previous outputs have reached the host (an event never recorded is
    // complete)
    SPIIR_CUDA_TRY(cudaStreamWaitEvent(s, p->copied[b], 0));
    SPIIR_CUDA_TRY(cudaMemcpyAsync(p->strain2[b], strain_host, sizeof(float) * nd * n, cudaMemcpyHostToDevice, s));
    SPIIR_TRY(pipe_run(p, p->strain2[b], n, n, p->ms2[b], p->am2[b], p->nl2[b], nullptr, s));
    SPIIR_CUDA_TRY(cudaEventRecord(p->computed[b], s));
    SPIIR_CUDA_TRY(cudaStreamWaitEvent(p->copy, p->computed[b], 0));
    SPIIR_CUDA_TRY(cudaMemcpyAsync(ms_host, p->ms2[b], sizeof(float) * T * n, cudaMemcpyDeviceToHost, p->copy));
    SPIIR_CUDA_TRY(cudaMemcpyAsync(am_host, p->am2[b], sizeof(int32_t) * T * n, cudaMemcpyDeviceToHost, p->copy));
    SPIIR_CUDA_TRY(cudaMemcpyAsync(nl_host, p->nl2[b], sizeof(float) * T * n, cudaMemcpyDeviceToHost, p->copy));
    SPIIR_CUDA_TRY(cudaEventRecord(p->copied[b], p->copy));
    p->abuf = 1 - b;
    return SPIIR_OK;
}

extern "C" int spiir_pipeline_wait(spiir_pipeline_t p) {
    clear_error();
    if (!p) return fail(SPIIR_EINVAL, "pipeline is NULL");
    if (p->async_ready) SPIIR_CUDA_TRY(cudaStreamSynchronize(p->copy));
    return SPIIR_OK;
}

extern "C" int spiir_pipeline_wait_for(spiir_pipeline_t p, double timeout_s) {
    clear_error();
    if (!p) return fail(SPIIR_EINVAL, "pipeline is NULL");
    if (!(timeout_s >= 0.0)) return fail(SPIIR_EINVAL, "timeout_s = %g", timeout_s);
    if (!p->async_ready) return SPIIR_OK;
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
    for (;;) {
        const cudaError_t e = cudaStreamQuery(p->copy);
        if (e == cudaSuccess) return SPIIR_OK;
        if (e != cudaErrorNotReady) {
            cudaGetLastError();
            return fail(SPIIR_ECUDA, "cudaStreamQuery failed: %s", cudaGetErrorString(e));
        }
        if (std::chrono::steady_clock::now() >= deadline)
            return fail(SPIIR_ETIMEOUT, "submitted steps not complete after %g s", timeout_s);
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}
