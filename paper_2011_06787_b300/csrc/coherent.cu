// Coherent all-sky scan (Sec. II.C.1 Eq. (llr_form), Eq. (null_def); App. A):
//     w_I(p, k) = z_I[k + Delta_I(p)]
//     rho_C^2(p, k) = sum_{j=1,2} | sum_I U_s[p][I][j] w_I |^2,   max and argmax over p,
//     null at the argmax = sum_{j>2} | sum_I U_null[p][I][j] w_I |^2.
//
// Device mapping (K2): a persistent grid walks work items (template, tile of KT output
// samples).  For each item the block stages the N_d SNR rows of the tile plus a halo of
// H samples on each side into shared memory; the per-pixel table (offsets H + Delta_I and
// the two signal columns of U) stays resident in shared memory for the whole launch when
// it fits, else it is read through L1.  A thread owns Q output samples, spaced by the
// block size so that every shared-memory load of a warp touches consecutive float2
// words, and loops over all pixels keeping a running maximum and the first pixel that
// attains it.  The null stream is evaluated once per sample at the winning pixel.
#include <algorithm>
#include <cmath>
#include <vector>

#include "coherent.cuh"

namespace spiir {

template <int ND>
struct __align__(16) TabEntry {
    float u[ND][2];
    short off[ND];
};

template <int ND, bool SMEM_TAB, bool MAP>
__global__ void __launch_bounds__(kCohThreads) k_coherent(const __grid_constant__ CohArgs a) {
    constexpr int Q = kCohQ;
    constexpr int KT = kCohThreads * Q;
    extern __shared__ __align__(16) unsigned char smem[];
    using Entry = TabEntry<ND>;
    const Entry *tab;
    float2 *zs;
    const int tid = threadIdx.x;
    const int W = KT + 2 * a.H;
    if (SMEM_TAB) {
        Entry *t = reinterpret_cast<Entry *>(smem);
        const uint4 *src = reinterpret_cast<const uint4 *>(a.table);
        uint4 *dst = reinterpret_cast<uint4 *>(t);
        const int nvec = a.n_pix * (int)(sizeof(Entry) / 16);
        for (int i = tid; i < nvec; i += kCohThreads) dst[i] = src[i];
        tab = t;
        zs = reinterpret_cast<float2 *>(smem + a.tab_bytes);
    } else {
        tab = reinterpret_cast<const Entry *>(a.table);
        zs = reinterpret_cast<float2 *>(smem);
    }
    const int ntiles = (int)((a.n + KT - 1) / KT);
    const int64_t n_items = (int64_t)a.n_templates * ntiles;
    for (int64_t item = blockIdx.x; item < n_items; item += gridDim.x) {
        const int t = (int)(item / ntiles);
        const int64_t k0 = (item % ntiles) * (int64_t)KT;
        __syncthreads();  // previous item done with zs (and the table is staged)
        for (int I = 0; I < ND; ++I) {
            const float2 *row = a.snr + ((int64_t)t * ND + I) * a.pitch + k0;
            const int64_t lim = a.n + 2 * a.H - k0;  // valid entries of this row from k0
            for (int j = tid; j < W; j += kCohThreads) zs[I * W + j] = (j < lim) ? row[j] : make_float2(0.f, 0.f);
        }
        __syncthreads();
        float best[Q];
        int arg[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            best[q] = -1.0f;
            arg[q] = 0;
        }
#pragma unroll 2
        for (int p = 0; p < a.n_pix; ++p) {
            const Entry e = tab[p];
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                const int k = tid + q * kCohThreads;
                float y0r = 0.f, y0i = 0.f, y1r = 0.f, y1i = 0.f;
#pragma unroll
                for (int I = 0; I < ND; ++I) {
                    const float2 w = zs[I * W + e.off[I] + k];
                    y0r = fmaf(e.u[I][0], w.x, y0r);
                    y0i = fmaf(e.u[I][0], w.y, y0i);
                    y1r = fmaf(e.u[I][1], w.x, y1r);
                    y1i = fmaf(e.u[I][1], w.y, y1i);
                }
                const float v = fmaf(y1i, y1i, fmaf(y1r, y1r, fmaf(y0i, y0i, y0r * y0r)));
                if (MAP && k0 + k < a.n) a.skymap[((int64_t)t * a.n_pix + p) * a.n + k0 + k] = v;
                if (v > best[q]) {
                    best[q] = v;
                    arg[q] = p;
                }
            }
        }
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int k = tid + q * kCohThreads;
            if (k0 + k >= a.n) continue;
            float nul = 0.f;
            if (ND > 2) {
                const Entry e = tab[arg[q]];
                const float *un = a.u_null + (int64_t)arg[q] * ND * (ND - 2);
                for (int j = 0; j < ND - 2; ++j) {
                    float cr = 0.f, ci = 0.f;
                    for (int I = 0; I < ND; ++I) {
                        const float2 w = zs[I * W + e.off[I] + k];
                        const float u = un[I * (ND - 2) + j];
                        cr = fmaf(u, w.x, cr);
                        ci = fmaf(u, w.y, ci);
                    }
                    nul = fmaf(cr, cr, fmaf(ci, ci, nul));
                }
            }
            const int64_t o = (int64_t)t * a.n + k0 + k;
            a.max_stat[o] = best[q];
            a.argmax[o] = arg[q];
            a.null_stat[o] = nul;
        }
    }
}

template <int ND, bool SMEM_TAB, bool MAP>
static int launch_coh(const CohArgs &a, size_t smem, cudaStream_t stream) {
    auto kern = k_coherent<ND, SMEM_TAB, MAP>;
    static int blocks_per_sm[2] = {-1, -1};
    static size_t smem_seen[2] = {0, 0};
    int dev = 0;
    SPIIR_CUDA_TRY(cudaGetDevice(&dev));
    const int slot = 0;
    if (blocks_per_sm[slot] < 0 || smem_seen[slot] != smem) {
        SPIIR_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
        int nb = 0;
        SPIIR_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, kCohThreads, smem));
        blocks_per_sm[slot] = std::max(1, nb);
        smem_seen[slot] = smem;
    }
    int n_sm = 0;
    SPIIR_CUDA_TRY(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
    const int KT = kCohThreads * kCohQ;
    const int64_t items = (int64_t)a.n_templates * ((a.n + KT - 1) / KT);
    const int grid = (int)std::min<int64_t>(items, (int64_t)n_sm * blocks_per_sm[slot]);
    kern<<<grid, kCohThreads, smem, stream>>>(a);
    SPIIR_CUDA_TRY(cudaGetLastError());
    return SPIIR_OK;
}

template <int ND>
static int dispatch_nd(const CohArgs &a, bool smem_tab, bool map, size_t smem, cudaStream_t s) {
    if (smem_tab) return map ? launch_coh<ND, true, true>(a, smem, s) : launch_coh<ND, true, false>(a, smem, s);
    return map ? launch_coh<ND, false, true>(a, smem, s) : launch_coh<ND, false, false>(a, smem, s);
}

int coherent_scan(spiir_sky_s *sky, const float2 *snr, int64_t pitch, int T, int64_t n, float *max_stat,
                  int32_t *argmax, float *null_stat, float *skymap, cudaStream_t stream) {
    CohArgs a{};
    a.snr = snr;
    a.pitch = pitch;
    a.n_templates = T;
    a.n = n;
    a.H = sky->halo;
    a.n_pix = sky->n_pix;
    a.table = sky->table;
    a.u_null = sky->u_null;
    a.max_stat = max_stat;
    a.argmax = argmax;
    a.null_stat = null_stat;
    a.skymap = skymap;
    const int KT = kCohThreads * kCohQ;
    const size_t zbytes = (size_t)sky->n_det * (KT + 2 * sky->halo) * sizeof(float2);
    const bool smem_tab = sky->table_bytes + zbytes <= (size_t)kCohSmemTableLimit;
    a.tab_bytes = smem_tab ? sky->table_bytes : 0;
    const size_t smem = a.tab_bytes + zbytes;
    const bool map = skymap != nullptr;
    switch (sky->n_det) {
        case 2: return dispatch_nd<2>(a, smem_tab, map, smem, stream);
        case 3: return dispatch_nd<3>(a, smem_tab, map, smem, stream);
        case 4: return dispatch_nd<4>(a, smem_tab, map, smem, stream);
        default: return fail(SPIIR_EUNSUPPORTED, "n_det = %d", sky->n_det);
    }
}

template <int ND>
static void build_table(spiir_sky_s *s, const int32_t *delays, const float *u_sig) {
    std::vector<TabEntry<ND>> t(s->n_pix);
    for (int p = 0; p < s->n_pix; ++p) {
        TabEntry<ND> e{};
        for (int I = 0; I < ND; ++I) {
            e.u[I][0] = u_sig[((int64_t)p * ND + I) * 2];
            e.u[I][1] = u_sig[((int64_t)p * ND + I) * 2 + 1];
            e.off[I] = (short)(s->halo + delays[(int64_t)p * ND + I]);
        }
        t[p] = e;
    }
    s->h_table.resize(t.size() * sizeof(TabEntry<ND>));
    memcpy(s->h_table.data(), t.data(), s->h_table.size());
}

}  // namespace spiir

using namespace spiir;

static void sky_free(spiir_sky_s *s) {
    if (!s) return;
    dev_free(s->table);
    dev_free(s->u_null);
    delete s;
}

extern "C" int spiir_sky_create(int n_det, int n_pix, const int32_t *delays, const float *u_sig,
                                const float *u_null, spiir_sky_t *out) {
    clear_error();
    if (!out) return fail(SPIIR_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_det < 2 || n_det > 4) return fail(SPIIR_EINVAL, "n_det = %d outside [2, 4]", n_det);
    if (n_pix < 1 || n_pix > (1 << 20)) return fail(SPIIR_EINVAL, "n_pix = %d outside [1, 2^20]", n_pix);
    if (!delays || !u_sig || (n_det > 2 && !u_null)) return fail(SPIIR_EINVAL, "NULL table pointer");
    int H = 0;
    for (int64_t i = 0; i < (int64_t)n_pix * n_det; ++i) {
        if (delays[i] < -kCohMaxHalo || delays[i] > kCohMaxHalo)
            return fail(SPIIR_EINVAL, "delay %d outside [-%d, %d]", delays[i], kCohMaxHalo, kCohMaxHalo);
        H = std::max(H, std::abs(delays[i]));
    }
    for (int64_t i = 0; i < (int64_t)n_pix * n_det * 2; ++i)
        if (!std::isfinite(u_sig[i])) return fail(SPIIR_EINVAL, "u_sig holds a non-finite value");
    if (n_det > 2)
        for (int64_t i = 0; i < (int64_t)n_pix * n_det * (n_det - 2); ++i)
            if (!std::isfinite(u_null[i])) return fail(SPIIR_EINVAL, "u_null holds a non-finite value");
    spiir_sky_s *s = new (std::nothrow) spiir_sky_s();
    if (!s) return fail(SPIIR_ENOMEM, "host allocation of the sky failed");
    s->n_det = n_det;
    s->n_pix = n_pix;
    s->halo = H;
    switch (n_det) {
        case 2: build_table<2>(s, delays, u_sig); break;
        case 3: build_table<3>(s, delays, u_sig); break;
        default: build_table<4>(s, delays, u_sig); break;
    }
    s->table_bytes = s->h_table.size();
    int rc = dev_alloc(&s->table, s->table_bytes, "sky table");
    if (rc == SPIIR_OK && cudaMemcpy(s->table, s->h_table.data(), s->table_bytes, cudaMemcpyHostToDevice) != cudaSuccess)
        rc = fail(SPIIR_ECUDA, "copy of the sky table failed");
    if (rc == SPIIR_OK && n_det > 2) {
        const size_t nb = sizeof(float) * n_pix * n_det * (n_det - 2);
        rc = dev_alloc((void **)&s->u_null, nb, "null-space table");
        if (rc == SPIIR_OK && cudaMemcpy(s->u_null, u_null, nb, cudaMemcpyHostToDevice) != cudaSuccess)
            rc = fail(SPIIR_ECUDA, "copy of the null-space table failed");
    }
    if (rc != SPIIR_OK) {
        sky_free(s);
        return rc;
    }
    *out = s;
    return SPIIR_OK;
}

extern "C" void spiir_sky_destroy(spiir_sky_t s) { sky_free(s); }

extern "C" int spiir_sky_info(spiir_sky_t s, int *n_det, int *n_pix, int *halo) {
    if (!s) return fail(SPIIR_EINVAL, "sky is NULL");
    if (n_det) *n_det = s->n_det;
    if (n_pix) *n_pix = s->n_pix;
    if (halo) *halo = s->halo;
    return SPIIR_OK;
}

extern "C" int spiir_coherent_scan(spiir_sky_t s, const float *snr, int64_t pitch, int T, int64_t n,
                                   float *max_stat, int32_t *argmax, float *null_stat, float *skymap,
                                   void *stream) {
    clear_error();
    if (!s) return fail(SPIIR_EINVAL, "sky is NULL");
    if (!snr || !max_stat || !argmax || !null_stat) return fail(SPIIR_EINVAL, "NULL buffer");
    if (T < 1 || n < 1) return fail(SPIIR_EINVAL, "n_templates = %d, n = %lld", T, (long long)n);
    if (pitch < n + 2 * s->halo)
        return fail(SPIIR_EINVAL, "snr_pitch %lld < n + 2 H = %lld", (long long)pitch, (long long)(n + 2 * s->halo));
    if (((uintptr_t)snr) % 8 != 0) return fail(SPIIR_EINVAL, "snr pointer is not 8-byte aligned");
    return coherent_scan(s, reinterpret_cast<const float2 *>(snr), pitch, T, n, max_stat, argmax, null_stat,
                         skymap, (cudaStream_t)stream);
}
