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
#include <cstdlib>
#include <vector>

#include "coherent.cuh"

namespace spiir {

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

// ---------------------------------------------------------------------------------------
// Grouped scan for 2 and 3 detectors.
//
// For N_d = 3 the signal plane and the unit null vector n(p) complete each other
// (U_s U_s^T + n n^T = I), so rho_C^2 = |w|^2 - |n.w|^2 and the null stream at p is
// |n.w|^2 (App. A, Eq. (null_def)).  For N_d = 2 rho_C^2 = |w|^2 and the null is 0.
// Pixels are visited sorted by (Delta_0, Delta_1, Delta_2), grouped by Delta_0, so the SNR of
// detector 0 and its power are loaded once per group.  The SNR tile is kept in shared memory as
// separate real and imaginary planes, each twice (shifted by one sample), so a thread loads
// the pair (z[k + off], z[k + 1 + off]) for any offset with one aligned 8-byte access and
// evaluates two samples with packed f32x2 arithmetic.  The inner loop keeps only a running
// maximum per group; after all groups, each sample rescans its winning group with the same
// arithmetic in scalar form to find the lowest pixel index that attains the maximum (a full
// rescan if two groups tie exactly).

__device__ __forceinline__ u64 lds64(const float *p) { return *reinterpret_cast<const u64 *>(p); }

// one sample in scalar form: the same IEEE operations in the same order as the packed loop
template <int ND>
__device__ __forceinline__ void stat_one(const float *pl, int W, int i0, int i1, int i2, float n0, float n1, float n2,
                                         int k, float &v, float &t) {
    const float w0r = pl[i0 + k], w0i = pl[i0 + 2 * W + k];
    const float w1r = pl[i1 + k], w1i = pl[i1 + 2 * W + k];
    const float s0 = __fmaf_rn(w0r, w0r, __fmul_rn(w0i, w0i));
    float S = __fmaf_rn(w1i, w1i, __fmaf_rn(w1r, w1r, s0));
    if (ND == 3) {
        const float w2r = pl[i2 + k], w2i = pl[i2 + 2 * W + k];
        const float nr = __fmaf_rn(n2, w2r, __fmaf_rn(n1, w1r, __fmul_rn(n0, w0r)));
        const float ni = __fmaf_rn(n2, w2i, __fmaf_rn(n1, w1i, __fmul_rn(n0, w0i)));
        S = __fmaf_rn(w2i, w2i, __fmaf_rn(w2r, w2r, S));
        t = __fmaf_rn(ni, ni, __fmul_rn(nr, nr));
        v = __fmaf_rn(t, -1.f, S);
    } else {
        t = 0.f;
        v = S;
    }
}

template <int ND, bool TAB_SMEM, bool MAP, int TPB, int PPT>
__global__ void __launch_bounds__(TPB) k_coherent_grouped(const __grid_constant__ GroupedArgs a) {
    constexpr int KT = 2 * TPB * PPT;   // output samples per work item
    constexpr int NQ = 2 * PPT;         // samples per thread
    extern __shared__ __align__(16) unsigned char smem[];
    const int tid = threadIdx.x;
    const int P = a.n_pix, G = a.n_grp, W = a.W;
    size_t off = 0;
    const float4 *ent;
    if (TAB_SMEM) {
        float4 *e = reinterpret_cast<float4 *>(smem);
        for (int i = tid; i < P; i += TPB) e[i] = a.ent[i];
        ent = e;
        off = (size_t)P * sizeof(float4);
    } else {
        ent = a.ent;
    }
    uint16_t *orig = reinterpret_cast<uint16_t *>(smem + off);
    for (int i = tid; i < P; i += TPB) orig[i] = a.orig[i];
    off += ((size_t)P * sizeof(uint16_t) + 15) / 16 * 16;
    int4 *grp = reinterpret_cast<int4 *>(smem + off);
    for (int i = tid; i < G; i += TPB) grp[i] = a.grp[i];
    off += (size_t)G * sizeof(int4);
    float *pl = reinterpret_cast<float *>(smem + off);

    const int ntiles = (int)((a.n + KT - 1) / KT);
    const int64_t n_items = (int64_t)a.n_templates * ntiles;
    for (int64_t item = blockIdx.x; item < n_items; item += gridDim.x) {
        const int t = (int)(item / ntiles);
        const int64_t k0 = (item % ntiles) * (int64_t)KT;
        __syncthreads();
        for (int I = 0; I < ND; ++I) {
            const float2 *row = a.snr + ((int64_t)t * ND + I) * a.pitch + k0;
            const int64_t lim = a.n + 2 * a.H - k0;
            float *b = pl + I * 4 * W;
            for (int j = tid; j < W; j += TPB) {
#ifdef SPIIR_CHECKED
                if (j < lim && k0 + j >= a.pitch) {
                    report_bounds(a.status, 30);
                    continue;
                }
#endif
                const float2 v = (j < lim) ? row[j] : make_float2(0.f, 0.f);
                b[j] = v.x;
                b[2 * W + j] = v.y;
                if (j > 0) {
                    b[W + j - 1] = v.x;
                    b[3 * W + j - 1] = v.y;
                } else {
                    b[2 * W - 1] = 0.f;
                    b[4 * W - 1] = 0.f;
                }
            }
        }
        __syncthreads();
        // per sample: the maximum, the first group attaining it, the second one (tie bit set),
        // and whether a third one does (multi bit set)
        float best[NQ];
        int bg[NQ], bg2[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            best[q] = -INFINITY;
            bg[q] = 0;
            bg2[q] = 0;
        }
        unsigned tie = 0, multi = 0;
        for (int g = 0; g < G; ++g) {
            const int4 gr = grp[g];
            u64 w0r[PPT], w0i[PPT], s0[PPT];
            float gm[NQ];
#pragma unroll
            for (int h = 0; h < PPT; ++h) {
                const int k = 2 * tid + h * 2 * TPB;
                w0r[h] = lds64(pl + gr.x + k);
                w0i[h] = lds64(pl + gr.x + 2 * W + k);
                s0[h] = fma2(w0r[h], w0r[h], mul2(w0i[h], w0i[h]));
                gm[2 * h] = -INFINITY;
                gm[2 * h + 1] = -INFINITY;
            }
            // Software pipeline over the pixels of the group: while pixel p is evaluated, the SNR
            // loads of pixel p + 1 are in flight and the table entry of pixel p + 2 is fetched.
            // Indices are clamped at the end of the group (the extra loads are discarded).
            const int p0 = gr.y, p1 = gr.z;
            float4 e = TAB_SMEM ? ent[p0] : __ldg(&ent[p0]);
            float4 en = TAB_SMEM ? ent[min(p0 + 1, p1 - 1)] : __ldg(&ent[min(p0 + 1, p1 - 1)]);
            u64 a1r[PPT], a1i[PPT], a2r[PPT], a2i[PPT];
            {
                const unsigned o = __float_as_uint(e.w);
                const int i1 = (int)(o & 0x7FFFu), i2 = (int)(o >> 16);
#pragma unroll
                for (int h = 0; h < PPT; ++h) {
                    const int k = 2 * tid + h * 2 * TPB;
                    a1r[h] = lds64(pl + i1 + k);
                    a1i[h] = lds64(pl + i1 + 2 * W + k);
                    if (ND == 3) {
                        a2r[h] = lds64(pl + i2 + k);
                        a2i[h] = lds64(pl + i2 + 2 * W + k);
                    }
                }
            }
#pragma unroll 2
            for (int p = p0; p < p1; ++p) {
                // loads of the next pixel
                u64 b1r[PPT], b1i[PPT], b2r[PPT], b2i[PPT];
                {
                    const unsigned o = __float_as_uint(en.w);
                    const int i1 = (int)(o & 0x7FFFu), i2 = (int)(o >> 16);
#pragma unroll
                    for (int h = 0; h < PPT; ++h) {
                        const int k = 2 * tid + h * 2 * TPB;
                        b1r[h] = lds64(pl + i1 + k);
                        b1i[h] = lds64(pl + i1 + 2 * W + k);
                        if (ND == 3) {
                            b2r[h] = lds64(pl + i2 + k);
                            b2i[h] = lds64(pl + i2 + 2 * W + k);
                        }
                    }
                }
                const int pnn = min(p + 2, p1 - 1);
                const float4 enn = TAB_SMEM ? ent[pnn] : __ldg(&ent[pnn]);
                // evaluate pixel p
#pragma unroll
                for (int h = 0; h < PPT; ++h) {
                    const u64 s01 = fma2(a1i[h], a1i[h], fma2(a1r[h], a1r[h], s0[h]));
                    u64 v;
                    if (ND == 3) {
                        const u64 N0 = pack2(e.x, e.x), N1 = pack2(e.y, e.y), N2 = pack2(e.z, e.z);
                        const u64 nr = fma2(N2, a2r[h], fma2(N1, a1r[h], mul2(N0, w0r[h])));
                        const u64 ni = fma2(N2, a2i[h], fma2(N1, a1i[h], mul2(N0, w0i[h])));
                        const u64 S = fma2(a2i[h], a2i[h], fma2(a2r[h], a2r[h], s01));
                        const u64 t = fma2(ni, ni, mul2(nr, nr));
                        v = fma2(t, pack2(-1.f, -1.f), S);
                    } else {
                        v = s01;
                    }
                    const float2 f = unpack2(v);
                    if (MAP) {
                        const int k = 2 * tid + h * 2 * TPB;
                        float *mrow = a.skymap + ((int64_t)t * P + orig[p]) * a.n + k0;
                        if (k0 + k < a.n) mrow[k] = f.x;
                        if (k0 + k + 1 < a.n) mrow[k + 1] = f.y;
                    }
                    gm[2 * h] = fmaxf(gm[2 * h], f.x);
                    gm[2 * h + 1] = fmaxf(gm[2 * h + 1], f.y);
                }
#pragma unroll
                for (int h = 0; h < PPT; ++h) {
                    a1r[h] = b1r[h];
                    a1i[h] = b1i[h];
                    if (ND == 3) {
                        a2r[h] = b2r[h];
                        a2i[h] = b2i[h];
                    }
                }
                e = en;
                en = enn;
            }
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                if (gm[q] > best[q]) {
                    best[q] = gm[q];
                    bg[q] = g;
                    tie &= ~(1u << q);
                    multi &= ~(1u << q);
                } else if (gm[q] == best[q]) {
                    if (tie >> q & 1u) multi |= 1u << q;
                    bg2[q] = g;
                    tie |= 1u << q;
                }
            }
        }
        // resolve the argmax (lowest original pixel index among equal maxima) and the null
        for (int q = 0; q < NQ; ++q) {
            const int k = 2 * tid + (q >> 1) * 2 * TPB + (q & 1);
            if (k0 + k >= a.n) continue;
            int arg = 0x7fffffff;
            float nul = 0.f;
            int g_lo = bg[q], g_hi = bg[q] + 1, g_two = -1;
            if (tie >> q & 1u) {
                // equal maxima in different groups: pixel 0, the lowest index, wins if it
                // attains the maximum (the all-zero window); otherwise the two groups that attain
                // it are rescanned, or every group when a third one does too
                const float4 e = ent[a.q0];
                const unsigned o = __float_as_uint(e.w);
                float v, tt;
                stat_one<ND>(pl, W, grp[a.g0].x, (int)(o & 0x7FFFu), (int)(o >> 16), e.x, e.y, e.z, k, v, tt);
                if (v == best[q]) {
                    arg = 0;
                    nul = tt;
                    g_hi = g_lo;
                } else if (multi >> q & 1u) {
                    g_lo = 0;
                    g_hi = G;
                } else {
                    g_two = bg2[q];
                }
            }
            for (int gi = g_lo; gi < g_hi + (g_two >= 0); ++gi) {
                const int g = gi < g_hi ? gi : g_two;
                const int4 gr = grp[g];
                for (int p = gr.y; p < gr.z; ++p) {
                    const float4 e = ent[p];
                    const unsigned o = __float_as_uint(e.w);
                    float v, tt;
                    stat_one<ND>(pl, W, gr.x, (int)(o & 0x7FFFu), (int)(o >> 16), e.x, e.y, e.z, k, v, tt);
                    const int op = orig[p];
                    if (v == best[q] && op < arg) {
                        arg = op;
                        nul = tt;
                    }
                }
            }
            if (arg == 0x7fffffff) arg = 0;  // only when every statistic is NaN
            const int64_t o = (int64_t)t * a.n + k0 + k;
#ifdef SPIIR_CHECKED
            if (o >= (int64_t)a.n_templates * a.n || arg < 0 || arg >= P) {
                report_bounds(a.status, 31);
                continue;
            }
#endif
            a.max_stat[o] = best[q];
            a.argmax[o] = arg;
            a.null_stat[o] = nul;
        }
    }
}

template <int ND, bool TAB_SMEM, bool MAP, int TPB, int PPT>
static int launch_grouped(const GroupedArgs &a, size_t smem, cudaStream_t stream) {
    auto kern = k_coherent_grouped<ND, TAB_SMEM, MAP, TPB, PPT>;
    SPIIR_TRY(set_max_dyn_smem((const void *)kern, 227 * 1024));
    int blocks_per_sm = 0;
    SPIIR_TRY(resident_blocks_per_sm((const void *)kern, TPB, smem, &blocks_per_sm));
    blocks_per_sm = std::max(1, blocks_per_sm);
    int dev = 0, n_sm = 0;
    SPIIR_CUDA_TRY(cudaGetDevice(&dev));
    SPIIR_CUDA_TRY(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
    const int KT = 2 * TPB * PPT;
    const int64_t items = (int64_t)a.n_templates * ((a.n + KT - 1) / KT);
    const int grid = (int)std::min<int64_t>(items, (int64_t)n_sm * blocks_per_sm);
    kern<<<grid, TPB, smem, stream>>>(a);
    SPIIR_CUDA_TRY(cudaGetLastError());
    return SPIIR_OK;
}

template <int ND, int TPB, int PPT>
static int dispatch_grouped3(const GroupedArgs &a, bool tab_smem, bool map, size_t smem, cudaStream_t s) {
    if (tab_smem)
        return map ? launch_grouped<ND, true, true, TPB, PPT>(a, smem, s)
                   : launch_grouped<ND, true, false, TPB, PPT>(a, smem, s);
    return map ? launch_grouped<ND, false, true, TPB, PPT>(a, smem, s)
               : launch_grouped<ND, false, false, TPB, PPT>(a, smem, s);
}

template <int ND>
static int dispatch_grouped(const GroupedArgs &a, int tpb, int ppt, bool tab_smem, bool map, size_t smem,
                            cudaStream_t s) {
    if (tpb == 512 && ppt == 1) return dispatch_grouped3<ND, 512, 1>(a, tab_smem, map, smem, s);
    if (tpb == 256 && ppt == 1) return dispatch_grouped3<ND, 256, 1>(a, tab_smem, map, smem, s);
    if (tpb == 512 && ppt == 2) return dispatch_grouped3<ND, 512, 2>(a, tab_smem, map, smem, s);
    return dispatch_grouped3<ND, 256, 2>(a, tab_smem, map, smem, s);
}

template <int ND, bool SMEM_TAB, bool MAP>
static int launch_coh(const CohArgs &a, size_t smem, cudaStream_t stream) {
    auto kern = k_coherent<ND, SMEM_TAB, MAP>;
    SPIIR_TRY(set_max_dyn_smem((const void *)kern, 227 * 1024));
    int blocks_per_sm = 0;
    SPIIR_TRY(resident_blocks_per_sm((const void *)kern, kCohThreads, smem, &blocks_per_sm));
    blocks_per_sm = std::max(1, blocks_per_sm);
    int dev = 0, n_sm = 0;
    SPIIR_CUDA_TRY(cudaGetDevice(&dev));
    SPIIR_CUDA_TRY(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
    const int KT = kCohThreads * kCohQ;
    const int64_t items = (int64_t)a.n_templates * ((a.n + KT - 1) / KT);
    const int grid = (int)std::min<int64_t>(items, (int64_t)n_sm * blocks_per_sm);
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
    if (sky->grouped && sky->scan_tmem && sky->tmem_ok) {
        TmemArgs m{};
        m.snr = snr;
        m.pitch = pitch;
        m.n_templates = T;
        m.n = n;
        m.H = sky->halo;
        m.mw = sky->scan_tmem_mw;
        m.C = tmem_columns(sky->halo, m.mw);
        m.max_stat = max_stat;
        m.argmax = argmax;
        m.null_stat = null_stat;
        m.skymap = skymap;
        m.map_vec = (n % 4 == 0 && ((uintptr_t)skymap % 16) == 0) ? 1 : 0;
        m.sky_pix = sky->n_pix;
        // short chunks: several templates share a work item (their rows split the 128 lanes)
        m.nsub = tmem_templates_per_item(n, m.mw);
        for (size_t k = 0; k < sky->t_parts.size(); ++k) {
            const TmPart &pt = sky->t_parts[k];
            m.n_pix = pt.n_pix;
            m.ent = sky->t_ent + pt.first;
            m.orig = sky->g_orig + pt.first;
            m.grp = sky->t_grp + pt.gfirst;
            m.n_grp = pt.n_grp;
            m.q0 = pt.q0;
            m.g0 = pt.g0;
            for (int i = 0; i < 5; ++i) m.slice[i] = pt.slice[i];
            m.merge = k > 0 ? 1 : 0;
            SPIIR_TRY(launch_coherent_tmem(m, sky->scan_tmem_param ? pt.tab : nullptr, stream));
        }
        return SPIIR_OK;
    }
    if (sky->grouped) {
        GroupedArgs g{};
        g.snr = snr;
        g.pitch = pitch;
        g.n_templates = T;
        g.n = n;
        g.H = sky->halo;
        g.n_pix = sky->n_pix;
        g.ent = sky->g_ent;
        g.orig = sky->g_orig;
        g.grp = sky->g_grp;
        g.n_grp = sky->n_grp;
        g.q0 = sky->g_q0;
        g.g0 = sky->g_g0;
        g.W = sky->g_W;
        g.max_stat = max_stat;
        g.argmax = argmax;
        g.null_stat = null_stat;
        g.skymap = skymap;
        g.status = device_status_word();
        const int tpb = sky->scan_threads, ppt = sky->scan_pairs;
        g.W = 2 * tpb * ppt + 2 * sky->halo + 2;
        if (g.W != sky->g_W) return fail(SPIIR_EINVAL, "internal: plane length mismatch");
        const size_t fixed = ((size_t)sky->n_pix * sizeof(uint16_t) + 15) / 16 * 16 + (size_t)sky->n_grp * sizeof(int4) +
                             (size_t)sky->n_det * 4 * g.W * sizeof(float);
        const size_t tab = (size_t)sky->n_pix * sizeof(float4);
        const bool tab_smem = sky->scan_table_shared && fixed + tab <= (size_t)kCohSmemTableLimit;
        const size_t smem = fixed + (tab_smem ? tab : 0);
        if (sky->n_det == 3) return dispatch_grouped<3>(g, tpb, ppt, tab_smem, skymap != nullptr, smem, stream);
        return dispatch_grouped<2>(g, tpb, ppt, tab_smem, skymap != nullptr, smem, stream);
    }
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
    dev_free(s->g_ent);
    dev_free(s->g_orig);
    dev_free(s->g_grp);
    dev_free(s->t_ent);
    dev_free(s->d_delays);
    dev_free(s->pt_tab);
    dev_free(s->t_grp);
    for (auto &pt : s->t_parts) delete pt.tab;
    delete s;
}

// Grouped tables for 2 or 3 detectors, when the supplied U is an orthonormal basis whose
// signal plane has rank 2 (the null-vector form needs it); otherwise the general kernel runs.
static int build_grouped(spiir_sky_s *s, const int32_t *delays, const float *u_sig, const float *u_null) {
    const int nd = s->n_det, P = s->n_pix, H = s->halo;
    if (nd != 2 && nd != 3) return SPIIR_OK;
    if (P > 65535) return SPIIR_OK;
    for (int p = 0; p < P; ++p) {
        double U[3][3] = {{0}};
        for (int I = 0; I < nd; ++I) {
            U[I][0] = u_sig[((int64_t)p * nd + I) * 2];
            U[I][1] = u_sig[((int64_t)p * nd + I) * 2 + 1];
            if (nd == 3) U[I][2] = u_null[(int64_t)p * nd + I];
        }
        for (int i = 0; i < nd; ++i)
            for (int j = 0; j < nd; ++j) {
                double d = 0;
                for (int I = 0; I < nd; ++I) d += U[I][i] * U[I][j];
                if (std::fabs(d - (i == j ? 1.0 : 0.0)) > 1e-5) return SPIIR_OK;
            }
    }
    const int W = 2 * s->scan_threads * s->scan_pairs + 2 * H + 2;
    if (nd * 4 * W > 32767) return SPIIR_OK;  // plane indices use 15 bits
    std::vector<int> order(P);
    for (int p = 0; p < P; ++p) order[p] = p;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        for (int I = 0; I < nd; ++I) {
            const int dx = delays[(int64_t)x * nd + I], dy = delays[(int64_t)y * nd + I];
            if (dx != dy) return dx < dy;
        }
        return x < y;
    });
    auto plane_index = [&](int I, int delay) {
        const int o = H + delay, par = o & 1;
        return I * 4 * W + par * W + (o - par);
    };
    std::vector<float4> ent(P);
    std::vector<uint16_t> orig(P);
    std::vector<int4> grp;
    for (int q = 0; q < P; ++q) {
        const int p = order[q];
        const int d0 = delays[(int64_t)p * nd];
        if (grp.empty() || grp.back().w != d0) {
            if (!grp.empty()) grp.back().z = q;
            grp.push_back(make_int4(plane_index(0, d0), q, P, d0));
        }
        const unsigned i1 = (unsigned)plane_index(1, delays[(int64_t)p * nd + 1]);
        const unsigned i2 = nd == 3 ? (unsigned)plane_index(2, delays[(int64_t)p * nd + 2]) : 0u;
        float4 e;
        e.x = nd == 3 ? u_null[(int64_t)p * nd + 0] : 0.f;
        e.y = nd == 3 ? u_null[(int64_t)p * nd + 1] : 0.f;
        e.z = nd == 3 ? u_null[(int64_t)p * nd + 2] : 0.f;
        unsigned packed = i1 | (i2 << 16);
        memcpy(&e.w, &packed, 4);
        ent[q] = e;
        orig[q] = (uint16_t)p;
        if (p == 0) {
            s->g_q0 = q;
            s->g_g0 = (int)grp.size() - 1;
        }
    }
    SPIIR_TRY(dev_alloc((void **)&s->g_ent, sizeof(float4) * P, "grouped sky table"));
    SPIIR_TRY(dev_alloc((void **)&s->g_orig, sizeof(uint16_t) * P, "pixel order"));
    SPIIR_TRY(dev_alloc((void **)&s->g_grp, sizeof(int4) * grp.size(), "pixel groups"));
    SPIIR_CUDA_TRY(cudaMemcpy(s->g_ent, ent.data(), sizeof(float4) * P, cudaMemcpyHostToDevice));
    SPIIR_CUDA_TRY(cudaMemcpy(s->g_orig, orig.data(), sizeof(uint16_t) * P, cudaMemcpyHostToDevice));
    SPIIR_CUDA_TRY(cudaMemcpy(s->g_grp, grp.data(), sizeof(int4) * grp.size(), cudaMemcpyHostToDevice));
    s->n_grp = (int)grp.size();
    // tensor-memory scan: raw offsets delta_I = H + Delta_I; the groups cut into parts of at most
    // kTmTabPix pixels and kTmTabGrp groups, each part into four slices of consecutive groups
    // holding nearly equal numbers of pixels
    if (nd == 3 && 2 * tmem_columns(H, 8) <= 256) {
        std::vector<float4> te(ent);
        for (int q = 0; q < P; ++q) {
            const int p = order[q];
            const unsigned packed = (unsigned)(H + delays[(int64_t)p * nd + 1]) | ((unsigned)(H + delays[(int64_t)p * nd + 2]) << 16);
            memcpy(&te[q].w, &packed, 4);
        }
        // the fewest parts of nearly equal pixel counts: cut at the group boundaries closest to
        // k P / n_parts, and take one part more while a part exceeds the table limits
        std::vector<TmPart> parts;
        for (int np = (P + kTmTabPix - 1) / kTmTabPix; np <= s->n_grp && parts.empty(); ++np) {
            std::vector<int> cut{0};
            for (int k = 1; k < np; ++k) {
                const int64_t target = (int64_t)P * k / np;
                int best = cut.back() + 1;
                int64_t best_d = INT64_MAX;
                for (int c = cut.back() + 1; c < s->n_grp; ++c) {
                    const int64_t d = std::llabs((int64_t)grp[c].y - target);
                    if (d < best_d) {
                        best_d = d;
                        best = c;
                    }
                }
                cut.push_back(std::min(best, s->n_grp));
            }
            cut.push_back(s->n_grp);
            bool fits = true;
            for (int k = 0; k < np && fits; ++k) {
                TmPart pt;
                pt.gfirst = cut[k];
                pt.n_grp = cut[k + 1] - cut[k];
                if (pt.n_grp <= 0) {
                    fits = false;
                    break;
                }
                pt.first = grp[pt.gfirst].y;
                pt.n_pix = grp[cut[k + 1] - 1].z - pt.first;
                fits = pt.n_pix <= kTmTabPix && pt.n_grp <= kTmTabGrp;
                parts.push_back(pt);
            }
            if (!fits) parts.clear();
        }
        std::vector<int4> rg(grp);
        bool ok = !parts.empty();
        for (auto &pt : parts) {
            for (int g = pt.gfirst; g < pt.gfirst + pt.n_grp; ++g) {
                rg[g].y -= pt.first;
                rg[g].z -= pt.first;
            }
            // slices: the group boundary closest to each quarter of the part's pixels
            pt.slice[0] = 0;
            for (int k = 1; k < 4; ++k) {
                const int64_t target = (int64_t)pt.n_pix * k / 4;
                int best = pt.slice[k - 1];
                int64_t best_d = INT64_MAX;
                for (int c = pt.slice[k - 1]; c <= pt.n_grp; ++c) {
                    const int64_t start = c < pt.n_grp ? rg[pt.gfirst + c].y : pt.n_pix;
                    const int64_t d = start > target ? start - target : target - start;
                    if (d < best_d) {
                        best_d = d;
                        best = c;
                    }
                }
                pt.slice[k] = best;
            }
            pt.slice[4] = pt.n_grp;
            // the part's lowest pixel index and its group
            int qmin = 0;
            for (int q = 1; q < pt.n_pix; ++q)
                if (orig[pt.first + q] < orig[pt.first + qmin]) qmin = q;
            pt.q0 = qmin;
            for (int c = 0; c < pt.n_grp; ++c)
                if (rg[pt.gfirst + c].y <= qmin && qmin < rg[pt.gfirst + c].z) pt.g0 = c;
            pt.tab = new (std::nothrow) TmemTab();
            if (!pt.tab) {
                ok = false;
                break;
            }
            for (int q = 0; q < pt.n_pix; ++q) memcpy(&pt.tab->d12[q], &te[pt.first + q].w, 4);
            for (int c = 0; c < pt.n_grp; ++c) pt.tab->grp[c] = rg[pt.gfirst + c];
            ok = ok && tmem_fits(pt.n_pix, pt.n_grp, H, 8);
        }
        if (ok) {
            SPIIR_TRY(dev_alloc((void **)&s->t_ent, sizeof(float4) * P, "tensor-memory sky table"));
            SPIIR_CUDA_TRY(cudaMemcpy(s->t_ent, te.data(), sizeof(float4) * P, cudaMemcpyHostToDevice));
            SPIIR_TRY(dev_alloc((void **)&s->t_grp, sizeof(int4) * rg.size(), "tensor-memory pixel groups"));
            SPIIR_CUDA_TRY(cudaMemcpy(s->t_grp, rg.data(), sizeof(int4) * rg.size(), cudaMemcpyHostToDevice));
            s->t_parts = parts;
            s->tmem_ok = true;
        } else {
            for (auto &pt : parts) delete pt.tab;
        }
    }
    s->g_W = W;
    s->grouped = true;
    return SPIIR_OK;
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
    if (rc == SPIIR_OK) {
        s->h_delays.assign(delays, delays + (size_t)n_pix * n_det);
        std::vector<int16_t> d16(s->h_delays.begin(), s->h_delays.end());
        rc = dev_alloc((void **)&s->d_delays, sizeof(int16_t) * d16.size(), "sky delays");
        if (rc == SPIIR_OK && cudaMemcpy(s->d_delays, d16.data(), sizeof(int16_t) * d16.size(), cudaMemcpyHostToDevice) != cudaSuccess)
            rc = fail(SPIIR_ECUDA, "copy of the sky delays failed");
    }
    if (rc == SPIIR_OK) {
        s->h_usig.assign(u_sig, u_sig + (size_t)n_pix * n_det * 2);
        if (n_det > 2) s->h_unull.assign(u_null, u_null + (size_t)n_pix * n_det * (n_det - 2));
        rc = build_grouped(s, delays, u_sig, u_null);
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

extern "C" int spiir_sky_set_scan_shape(spiir_sky_t s, int threads, int pairs, int table_in_shared) {
    clear_error();
    if (!s) return fail(SPIIR_EINVAL, "sky is NULL");
    if ((threads == 512 || threads == 256) && pairs == 4) {
        // tensor-memory scan, 8 samples per thread row with 512 threads or 16 with 256; the
        // shared-memory kernel keeps its shape for sky-map requests
        const int mw = threads == 512 ? 8 : 16;
        bool fits = s->tmem_ok;
        for (const auto &pt : s->t_parts) fits = fits && tmem_fits(pt.n_pix, pt.n_grp, s->halo, mw);
        if (!fits)
            return fail(SPIIR_EUNSUPPORTED, "tensor-memory scan needs 3 detectors, an orthonormal basis, "
                                            "|Delta| <= %d and a table that fits in shared memory", mw == 8 ? 60 : 56);
        if (table_in_shared != 0 && table_in_shared != 1)
            return fail(SPIIR_EINVAL, "the third value of the tensor-memory shape must be 0 or 1");
        s->scan_tmem = 1;
        s->scan_tmem_param = table_in_shared;
        s->scan_tmem_mw = mw;
        return SPIIR_OK;
    }
    if ((threads != 256 && threads != 512) || (pairs != 1 && pairs != 2) || (table_in_shared != 0 && table_in_shared != 1))
        return fail(SPIIR_EINVAL, "threads must be 256 or 512, pairs 1, 2 or 4 (tensor memory), table_in_shared 0 or 1");
    s->scan_tmem = 0;
    s->scan_table_shared = table_in_shared;
    if (!s->grouped) {
        s->scan_threads = threads;
        s->scan_pairs = pairs;
        return SPIIR_OK;
    }
    const int ot = s->scan_threads, op = s->scan_pairs;
    SPIIR_CUDA_TRY(cudaDeviceSynchronize());
    dev_free(s->g_ent);
    dev_free(s->g_orig);
    dev_free(s->g_grp);
    dev_free(s->t_ent);
    dev_free(s->t_grp);
    for (auto &pt : s->t_parts) delete pt.tab;
    s->t_parts.clear();
    s->t_grp = nullptr;
    s->g_ent = nullptr;
    s->g_orig = nullptr;
    s->g_grp = nullptr;
    s->t_ent = nullptr;
    s->tmem_ok = false;
    s->grouped = false;
    s->scan_threads = threads;
    s->scan_pairs = pairs;
    int rc = build_grouped(s, s->h_delays.data(), s->h_usig.data(), s->n_det > 2 ? s->h_unull.data() : nullptr);
    if (rc != SPIIR_OK || !s->grouped) {
        s->scan_threads = ot;
        s->scan_pairs = op;
        build_grouped(s, s->h_delays.data(), s->h_usig.data(), s->n_det > 2 ? s->h_unull.data() : nullptr);
    }
    return rc;
}

extern "C" int spiir_sky_get_scan_shape(spiir_sky_t s, int *threads, int *pairs, int *table_in_shared, int *grouped) {
    if (!s) return fail(SPIIR_EINVAL, "sky is NULL");
    if (threads) *threads = s->scan_tmem ? (s->scan_tmem_mw == 16 ? 256 : 512) : s->scan_threads;
    if (pairs) *pairs = s->scan_tmem ? 4 : s->scan_pairs;
    if (table_in_shared) *table_in_shared = s->scan_tmem ? s->scan_tmem_param : s->scan_table_shared;
    if (grouped) *grouped = s->grouped ? 1 : 0;
    return SPIIR_OK;
}
