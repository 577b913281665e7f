// Coherent sky scan for three detectors with the delay windows of detectors 1 and 2 held in
// tensor memory (TMEM).
//
// The statistic is the one of the grouped shared-memory scan (App. A, Eq. (null_def)):
//     rho_C^2(p, k) = |w|^2 - |n(p).w|^2,   null(p, k) = |n(p).w|^2,
//     w_I = z_I[k + Delta_I(p)]  (Sec. II.C.1),
// evaluated with packed (real, imaginary) pairs: with A = |w_0|^2 + |w_1|^2 + |w_2|^2 and
// n.w formed component-wise, rho_C^2 = (A_re - (n.w)_re^2) + (A_im - (n.w)_im^2).  The scalar
// rescan that resolves the argmax recomputes the statistic of the candidate pixels and takes
// the largest (lowest pixel index among equals).
//
// Why TMEM: in the shared-memory kernel every (pixel, sample) reads 16 bytes of detector 1
// and 2 SNR from shared memory, and shared-memory bandwidth (one 128-byte wavefront per clock
// per SM) bounds the scan below the FP32 rate.  Here each of the 128 TMEM lanes belongs to one
// thread row and holds, for detectors 1 and 2, the SNR window z_I[k_r + c] (c = 0 .. C-1) of
// the row's first sample k_r, real and imaginary parts in adjacent columns 2c and 2c + 1.  The
// 8 samples k_r + m of a row at delay offset delta sit at columns 2 (delta + m), so one
// warp-uniform column address serves all 32 rows of a warp for any pixel, and every sample is
// one aligned two-column load that lands as an FP32 pair.
//
// Work item: one template and 1024 output samples (for chunks of at most 512 or 256 samples,
// 2 or 4 templates whose thread rows split the 128 lanes, each with its own segment of the
// staged tile).  Block: 512 threads = 16 warps, one block
// per SM (shared memory above half the SM's capacity keeps a second block off the SM, so the
// 512-column TMEM allocation never waits).  Warp w reads TMEM lanes 32 (w % 4) .. + 31 (the
// quarter its hardware position allows) and evaluates pixel slice w / 4: the sorted pixel
// groups are cut into four slices of nearly equal pixel count.  Per sample the four slice
// maxima are merged in shared memory; the sample's winning group is then rescanned in scalar
// arithmetic to find the lowest pixel index attaining the maximum, as in the shared-memory
// kernel.  A maximum that several groups attain exactly (unless the lowest pixel, pixel 0 with
// the all-zero window, settles it) is left to a second pass in which a whole warp rescans the
// sky for that sample.  A sky above 4096 pixels or 512 groups runs as consecutive parts that fit
// those limits, one launch each: every part after the first replaces a stored result only by a
// larger maximum, or an equal one at a lower pixel index.
// In sky-map mode every row also writes its 8 statistics of each pixel to
// map[t][p][k] (two 16-byte streaming stores), which overlaps the map's HBM writes with the
// arithmetic.
//
// Addresses in uniform registers.  A tcgen05.ld takes its tensor-memory address from a uniform
// register.  When the pixel's offsets come from shared memory the compiler cannot prove them
// warp-uniform and moves each address into a uniform register separately (one R2UR per load,
// 16 per pixel).  For skies of at most 4096 pixels and 512 groups the group table and the
// packed offsets are therefore passed as a __grid_constant__ kernel parameter (24 KB): read
// with indices derived from the warp index, they land in uniform registers directly, which
// removes those moves (116.5 -> 101.8 instructions per warp-pixel on the online workload).
#include <algorithm>

#include "coherent.cuh"

namespace spiir {

constexpr int kTmRows = 128;                // TMEM lanes = thread rows
constexpr int kTmDet = 256;                 // TMEM columns per detector (2 detectors, 512 columns)
constexpr int kTmMinSmem = 120 * 1024;      // keeps a second block off the SM
// MW consecutive samples per thread row: 8 with 512 threads (4 pixel slices of 4 warps) or 16
// with 256 threads (2 slices), so that a work item covers 128 MW samples either way
constexpr int tm_threads(int MW) { return MW == 8 ? 512 : 256; }

__device__ __forceinline__ void tm_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tm_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Two-column TMEM load (real, imaginary) of sample K of the window at addr, for this warp's
// 32 lanes.  The column 2 K after addr is even whenever addr is.
template <int K, int MW>
__device__ __forceinline__ void tl2(u64 (&w)[MW], uint32_t addr) {
    uint32_t lo, hi;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0, %1}, [%2+%3];"
                 : "=r"(lo), "=r"(hi)
                 : "r"(addr), "n"(2 * K)
                 : "memory");
    asm("mov.b64 %0, {%1, %2};" : "=l"(w[K]) : "r"(lo), "r"(hi));
}

template <int MW>
__device__ __forceinline__ void tm_window(u64 (&w)[MW], uint32_t addr) {
    tl2<0>(w, addr), tl2<1>(w, addr), tl2<2>(w, addr), tl2<3>(w, addr);
    tl2<4>(w, addr), tl2<5>(w, addr), tl2<6>(w, addr), tl2<7>(w, addr);
    if constexpr (MW == 16) {
        tl2<8>(w, addr), tl2<9>(w, addr), tl2<10>(w, addr), tl2<11>(w, addr);
        tl2<12>(w, addr), tl2<13>(w, addr), tl2<14>(w, addr), tl2<15>(w, addr);
    }
}

// Completes every outstanding TMEM load of the thread; the empty statements after it pin the
// loaded registers behind the wait.
template <int MW>
__device__ __forceinline__ void tm_wait_ld(u64 (&a)[MW], u64 (&b)[MW]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int m = 0; m < MW; ++m) asm volatile("" : "+l"(a[m]), "+l"(b[m]));
}

__device__ __forceinline__ void tm_st8(uint32_t addr, const float (&v)[8]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(addr),
                 "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7])
                 : "memory");
}


// shared-memory SNR planes, transposed by 8: element x at (x % 8) * L + x / 8, so the 32 rows
// of a warp reading sample 8 r + c hit 32 consecutive words
__device__ __forceinline__ int tpos(int x, int L) { return (x & 7) * L + (x >> 3); }

// PT: the group table and the per-pixel offsets come from the kernel parameter pt (read with
// warp-uniform indices, so the tensor-memory addresses stay in uniform registers); otherwise
// from shared memory.
template <bool MAP, bool PT, int NSUB, int MW>
__device__ __forceinline__ void tmem_scan(const TmemArgs &a, const TmemTab *pt) {
    constexpr int NT = tm_threads(MW), SL = NT / 128, KT = kTmRows * MW;  // threads, slices, slots
    extern __shared__ __align__(16) unsigned char smem[];
    const int tid = threadIdx.x, lane = tid & 31;
    // with PT the broadcast tells the compiler that the warp index (and so every table index
    // derived from it) is warp-uniform
    const int warp = PT ? __shfl_sync(0xffffffffu, tid >> 5, 0) : tid >> 5;
    const int q = warp & 3, sl = warp >> 2;
    const int row = 32 * q + lane;
    const int P = a.n_pix, G = a.n_grp, H = a.H, C = a.C;
    // nsub templates per work item: template s of the item owns rows s RPT .. (s + 1) RPT - 1
    // and the tile segment s SEG .. s SEG + SEG - 1 (its MW RPT samples plus the C-sample halo)
    constexpr int nsub = NSUB, RPT = kTmRows / NSUB, KS = MW * RPT;
    const int SEG = KS + C;
    const int W0 = nsub * SEG;      // staged samples per plane
    const int L = W0 / 8 + 1;       // transposed plane stride (odd)
    const int PL = 8 * L;           // floats per staged plane
    const int rsub = row / RPT;                          // this thread row's template in an item
    const int rbase = rsub * SEG + MW * (row % RPT);     // tile position of the row's first sample

    float4 *ent = reinterpret_cast<float4 *>(smem);
    size_t off = (size_t)P * sizeof(float4);
    int4 *grp = reinterpret_cast<int4 *>(smem + off);
    off += (size_t)G * sizeof(int4);
    float *cb_best = reinterpret_cast<float *>(smem + off);
    off += (size_t)SL * KT * sizeof(float);
    unsigned *cb_grp = reinterpret_cast<unsigned *>(smem + off);
    off += (size_t)SL * KT * sizeof(unsigned);
    float *zp = reinterpret_cast<float *>(smem + off);  // [3 detectors][re, im][PL]
    off += (size_t)6 * PL * sizeof(float);
    uint16_t *orig = reinterpret_cast<uint16_t *>(smem + off);
    off += ((size_t)P * sizeof(uint16_t) + 15) / 16 * 16;
    int *tie_slots = reinterpret_cast<int *>(smem + off);  // slots left to pass 2 of the merge
    off += (size_t)KT * sizeof(int);
    int *n_tie = reinterpret_cast<int *>(smem + off);
    off += 16;
    uint32_t *slot = reinterpret_cast<uint32_t *>(smem + off);

    for (int i = tid; i < P; i += NT) {
        ent[i] = a.ent[i];
        orig[i] = a.orig[i];
    }
    for (int i = tid; i < G; i += NT) grp[i] = a.grp[i];
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                     "r"(512u)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tm_fence_before();
    __syncthreads();
    tm_fence_after();
    const uint32_t tbase = PT ? __shfl_sync(0xffffffffu, *slot, 0) : *slot;
    const uint32_t la = tbase + ((uint32_t)(32 * q) << 16);  // this warp's lane quarter
    // the host cuts the groups into 4 slices; with 2 slices each takes two of them
    const int g_lo = a.slice[sl * (4 / SL)], g_hi = a.slice[(sl + 1) * (4 / SL)];

    const int ntiles = (int)((a.n + KS - 1) / KS);
    const int64_t n_items = (int64_t)((a.n_templates + nsub - 1) / nsub) * ntiles;
    for (int64_t item = blockIdx.x; item < n_items; item += gridDim.x) {
        const int t0 = (int)(item / ntiles) * nsub;      // the item's first template
        const int64_t k0 = (item % ntiles) * (int64_t)KS;
        const int64_t lim = a.n + 2 * H - k0;  // staged entries past this are zero
        const int trow = t0 + rsub;                      // this row's template
        // the previous item's TMEM and shared-memory reads are complete past this point
        tm_fence_before();
        __syncthreads();
        tm_fence_after();
        if (tid == 0) *n_tie = 0;  // read again only after the barrier that ends the staging
        for (int I = 0; I < 3; ++I) {
            float *re = zp + (2 * I) * PL, *im = re + PL;
            for (int x = tid; x < W0; x += NT) {
                const int s = x / SEG, j = x - s * SEG;
                const int ts = t0 + s;
                const float2 v = (ts < a.n_templates && j < lim) ? a.snr[((int64_t)ts * 3 + I) * a.pitch + k0 + j]
                                                                 : make_float2(0.f, 0.f);
                re[tpos(x, L)] = v.x;
                im[tpos(x, L)] = v.y;
            }
        }
        __syncthreads();
        // TMEM windows: unit u = 0..3 is detector 1 + (u & 1), window half u >> 1; warp slice
        // sl fills units sl, sl + SL, ...; four samples (8 columns) per store
        for (int u = sl; u < 4; u += SL) {
            const int I = 1 + (u & 1);
            const float *re = zp + (2 * I) * PL, *im = re + PL;
            const uint32_t base = la + (uint32_t)((I - 1) * kTmDet);
            const int h = C / 2;
            for (int c0 = (u >> 1) * h; c0 < (u >> 1) * h + h; c0 += 4) {
                float v[8];
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    const int x = rbase + c0 + m;
                    v[2 * m] = re[tpos(x, L)];
                    v[2 * m + 1] = im[tpos(x, L)];
                }
                tm_st8(base + 2 * c0, v);
            }
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        tm_fence_before();
        __syncthreads();
        tm_fence_after();

        // running maximum and winning group of this thread's samples within its slice, kept in
        // shared memory at [slice][m][row] (updated once per group)
        float *my_best = cb_best + sl * KT + row;
        unsigned *my_grp = cb_grp + sl * KT + row;
#pragma unroll
        for (int m = 0; m < MW; ++m) {
            my_best[m * kTmRows] = -INFINITY;
            my_grp[m * kTmRows] = 0;
        }
        const float *z0r = zp, *z0i = zp + PL;
        for (int g = g_lo; g < g_hi; ++g) {
            const int4 gr = PT ? pt->grp[g] : grp[g];
            const int d0 = H + gr.w;
            u64 w0[MW], s0[MW];
            float gm[MW];
#pragma unroll
            for (int m = 0; m < MW; ++m) {
                const int x = rbase + d0 + m;
                w0[m] = pack2(z0r[tpos(x, L)], z0i[tpos(x, L)]);
                s0[m] = mul2(w0[m], w0[m]);
                gm[m] = -INFINITY;
            }
            for (int p = gr.y; p < gr.z; ++p) {
                const float4 e = ent[p];
                const uint32_t o = PT ? pt->d12[p] : __float_as_uint(e.w);
                u64 w1[MW], w2[MW];
                tm_window(w1, la + 2 * (o & 0xFFFFu));
                tm_window(w2, la + kTmDet + 2 * (o >> 16));
                tm_wait_ld(w1, w2);
                const u64 N0 = pack2(e.x, e.x), N1 = pack2(e.y, e.y), N2 = pack2(e.z, e.z);
                float v[MW];
#pragma unroll
                for (int m = 0; m < MW; ++m) {
                    const u64 A = fma2(w2[m], w2[m], fma2(w1[m], w1[m], s0[m]));
                    const u64 nw = fma2(N2, w2[m], fma2(N1, w1[m], mul2(N0, w0[m])));
                    const float2 d = unpack2(sub2(A, mul2(nw, nw)));
                    v[m] = __fadd_rn(d.x, d.y);
                    gm[m] = fmaxf(gm[m], v[m]);
                }
                if (MAP && trow < a.n_templates) {
                    // the row's MW samples of this pixel: one contiguous segment per warp, written
                    // with the streaming (evict-first) hint
                    const int64_t kr = k0 + MW * (row % RPT);
                    float *mrow = a.skymap + ((int64_t)trow * a.sky_pix + orig[p]) * a.n + kr;
                    if (a.map_vec && kr + MW <= a.n) {
#pragma unroll
                        for (int m = 0; m < MW; m += 4)
                            __stcs(reinterpret_cast<float4 *>(mrow + m), make_float4(v[m], v[m + 1], v[m + 2], v[m + 3]));
                    } else {
#pragma unroll
                        for (int m = 0; m < MW; ++m)
                            if (kr + m < a.n) __stcs(mrow + m, v[m]);
                    }
                }
            }
#pragma unroll
            for (int m = 0; m < MW; ++m) {
                const float b = my_best[m * kTmRows];
                if (gm[m] > b) {
                    my_best[m * kTmRows] = gm[m];
                    my_grp[m * kTmRows] = (unsigned)g;
                } else if (gm[m] == b) {
                    my_grp[m * kTmRows] |= 0x80000000u;  // another group of this slice attains the same maximum
                }
            }
        }
        __syncthreads();
        // merge the slices and resolve the argmax (lowest original pixel index among equal maxima)
        // slot j = MW row + m: template t0 + row / RPT, its sample k0 + MW (row % RPT) + m,
        // tile position xj; it sits at [m][row] of the slice maxima
        auto slot_of = [&](int j, int &jk, int &xj, int &tj, int &cj) {
            const int jr = j / MW, js = jr / RPT;
            jk = MW * (jr - js * RPT) + j % MW;
            xj = js * SEG + jk;
            tj = t0 + js;
            cj = (j % MW) * kTmRows + jr;
        };
        // the statistic of sorted pixel p (detector-0 offset d0) at tile position xj, recomputed
        // in scalar arithmetic, and its null stream
        auto stat = [&](int p, int d0, int xj, float &v, float &tt) {
            const float4 e = ent[p];
            const uint32_t o = __float_as_uint(e.w);
            const int d1 = (int)(o & 0xFFFFu), d2 = (int)(o >> 16);
            const float *r0 = zp, *r1 = zp + 2 * PL, *r2 = zp + 4 * PL;
            const float w0r = r0[tpos(xj + d0, L)], w0i = r0[PL + tpos(xj + d0, L)];
            const float w1r = r1[tpos(xj + d1, L)], w1i = r1[PL + tpos(xj + d1, L)];
            const float w2r = r2[tpos(xj + d2, L)], w2i = r2[PL + tpos(xj + d2, L)];
            const float Ar = __fmaf_rn(w2r, w2r, __fmaf_rn(w1r, w1r, __fmul_rn(w0r, w0r)));
            const float Ai = __fmaf_rn(w2i, w2i, __fmaf_rn(w1i, w1i, __fmul_rn(w0i, w0i)));
            const float nr = __fmaf_rn(e.z, w2r, __fmaf_rn(e.y, w1r, __fmul_rn(e.x, w0r)));
            const float ni = __fmaf_rn(e.z, w2i, __fmaf_rn(e.y, w1i, __fmul_rn(e.x, w0i)));
            tt = __fmaf_rn(ni, ni, __fmul_rn(nr, nr));
            v = __fadd_rn(__fsub_rn(Ar, __fmul_rn(nr, nr)), __fsub_rn(Ai, __fmul_rn(ni, ni)));
        };
        // the candidate pixel with the largest recomputed statistic, lowest index among equals
        // (the compiler may contract the packed multiply-subtract of the main loop, so its value
        // and the recomputed one can differ in the last bit)
        auto take = [&](float v, int op, float tt, float &bv, int &arg, float &nul) {
            if (v > bv || (v == bv && op < arg)) {
                bv = v;
                arg = op;
                nul = tt;
            }
        };
        auto store = [&](int tj, int jk, float B, int arg, float nul) {
            if (arg == 0x7fffffff) arg = 0;  // only when every statistic is NaN
            const int64_t o = (int64_t)tj * a.n + k0 + jk;
            if (a.merge) {
                // a later part of the sky: replace the stored result only by a larger maximum,
                // or an equal one at a lower pixel
                const float old = a.max_stat[o];
                if (!(B > old || (B == old && arg < a.argmax[o]))) return;
            }
            a.max_stat[o] = B;
            a.argmax[o] = arg;
            a.null_stat[o] = nul;
        };
        // pass 1, one thread per slot: a maximum attained by one group is resolved by rescanning
        // that group; one attained by several groups either by pixel 0 (the all-zero window) or,
        // else, by pass 2
        for (int j = tid; j < KT; j += NT) {
            int jk, xj, tj, cj;
            slot_of(j, jk, xj, tj, cj);
            if (tj >= a.n_templates || k0 + jk >= a.n) continue;
            float B = cb_best[cj];
            for (int s = 1; s < SL; ++s) B = fmaxf(B, cb_best[s * KT + cj]);
            int hits = 0;
            unsigned gsel = 0, tie = 0;
            for (int s = 0; s < SL; ++s) {
                if (cb_best[s * KT + cj] == B) {
                    ++hits;
                    gsel = cb_grp[s * KT + cj] & 0x7FFFFFFFu;
                    tie |= cb_grp[s * KT + cj] >> 31;
                }
            }
            int arg = 0x7fffffff;
            float nul = 0.f, bv = -INFINITY;
            if (hits > 1 || tie) {
                float v, tt;
                stat(a.q0, H + grp[a.g0].w, xj, v, tt);
                if (v == B) {
                    store(tj, jk, B, orig[a.q0], tt);  // the lowest pixel index of the (part of the) sky
                } else {
                    tie_slots[atomicAdd(n_tie, 1)] = j;
                }
                continue;
            }
            const int4 gr = grp[gsel];
            for (int p = gr.y; p < gr.z; ++p) {
                float v, tt;
                stat(p, H + gr.w, xj, v, tt);
                take(v, orig[p], tt, bv, arg, nul);
            }
            store(tj, jk, B, arg, nul);
        }
        __syncthreads();
        // pass 2, one warp per slot whose maximum several groups attain (exact FP32 ties between
        // the top pixels of two groups, of the order of once per few million samples of noise):
        // the lanes share the groups, and a butterfly combines their best pixels under the same
        // rule
        for (int e = warp; e < *n_tie; e += NT / 32) {
            const int j = tie_slots[e];
            int jk, xj, tj, cj;
            slot_of(j, jk, xj, tj, cj);
            float B = cb_best[cj];
            for (int s = 1; s < SL; ++s) B = fmaxf(B, cb_best[s * KT + cj]);
            int arg = 0x7fffffff;
            float nul = 0.f, bv = -INFINITY;
            for (int g = lane; g < G; g += 32) {
                const int4 gr = grp[g];
                for (int p = gr.y; p < gr.z; ++p) {
                    float v, tt;
                    stat(p, H + gr.w, xj, v, tt);
                    take(v, orig[p], tt, bv, arg, nul);
                }
            }
#pragma unroll
            for (int m = 16; m >= 1; m >>= 1) {
                const float ov = __shfl_xor_sync(0xffffffffu, bv, m);
                const int oa = __shfl_xor_sync(0xffffffffu, arg, m);
                const float on = __shfl_xor_sync(0xffffffffu, nul, m);
                take(ov, oa, on, bv, arg, nul);
            }
            if (lane == 0) store(tj, jk, B, arg, nul);
        }
    }
    tm_fence_before();
    __syncthreads();
    tm_fence_after();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(512u) : "memory");
}

template <bool MAP, int NSUB, int MW>
__global__ void __launch_bounds__(tm_threads(MW), 1) k_coherent_tmem(const __grid_constant__ TmemArgs a) {
    tmem_scan<MAP, false, NSUB, MW>(a, nullptr);
}

template <bool MAP, int NSUB, int MW>
__global__ void __launch_bounds__(tm_threads(MW), 1) k_coherent_tmem_pt(const __grid_constant__ TmemArgs a,
                                                                       const __grid_constant__ TmemTab pt) {
    tmem_scan<MAP, true, NSUB, MW>(a, &pt);
}

template <int NSUB, int MW>
static int launch_tmem_nsub(const TmemArgs &a, const TmemTab *tab, int grid, size_t smem, cudaStream_t stream) {
    constexpr int NT = tm_threads(MW);
    SPIIR_TRY(set_max_dyn_smem((const void *)k_coherent_tmem<false, NSUB, MW>, 227 * 1024));
    SPIIR_TRY(set_max_dyn_smem((const void *)k_coherent_tmem<true, NSUB, MW>, 227 * 1024));
    SPIIR_TRY(set_max_dyn_smem((const void *)k_coherent_tmem_pt<false, NSUB, MW>, 227 * 1024));
    SPIIR_TRY(set_max_dyn_smem((const void *)k_coherent_tmem_pt<true, NSUB, MW>, 227 * 1024));
    if (tab && a.n_pix <= kTmTabPix && a.n_grp <= kTmTabGrp) {
        if (a.skymap)
            k_coherent_tmem_pt<true, NSUB, MW><<<grid, NT, smem, stream>>>(a, *tab);
        else
            k_coherent_tmem_pt<false, NSUB, MW><<<grid, NT, smem, stream>>>(a, *tab);
    } else if (a.skymap) {
        k_coherent_tmem<true, NSUB, MW><<<grid, NT, smem, stream>>>(a);
    } else {
        k_coherent_tmem<false, NSUB, MW><<<grid, NT, smem, stream>>>(a);
    }
    SPIIR_CUDA_TRY(cudaGetLastError());
    return SPIIR_OK;
}

size_t tmem_scan_smem(int n_pix, int n_grp, int C, int nsub, int mw) {
    const int KT = kTmRows * mw, SL = tm_threads(mw) / 128;
    const int W0 = KT + nsub * C, L = W0 / 8 + 1;
    size_t s = (size_t)n_pix * sizeof(float4) + (size_t)n_grp * sizeof(int4) + (size_t)2 * SL * KT * sizeof(float) +
               (size_t)6 * 8 * L * sizeof(float) + ((size_t)n_pix * sizeof(uint16_t) + 15) / 16 * 16 +
               (size_t)KT * sizeof(int) + 16 + 16;
    return std::max(s, (size_t)kTmMinSmem);
}

int tmem_columns(int H, int mw) { return (2 * H + mw + 15) / 16 * 16; }

bool tmem_fits(int n_pix, int n_grp, int H, int mw) {
    // sized for four templates per work item (the largest staged tile)
    return 2 * tmem_columns(H, mw) <= kTmDet && tmem_scan_smem(n_pix, n_grp, tmem_columns(H, mw), 4, mw) <= 227 * 1024;
}

int tmem_templates_per_item(int64_t n, int mw) {
    const int64_t ks = (int64_t)kTmRows * mw;  // samples of a one-template item
    return n <= ks / 4 ? 4 : (n <= ks / 2 ? 2 : 1);
}

int launch_coherent_tmem(const TmemArgs &a, const TmemTab *tab, cudaStream_t stream) {
    if (a.nsub != 1 && a.nsub != 2 && a.nsub != 4) return fail(SPIIR_EINVAL, "templates per item = %d", a.nsub);
    if (a.mw != 8 && a.mw != 16) return fail(SPIIR_EINVAL, "samples per row = %d", a.mw);
    const size_t smem = tmem_scan_smem(a.n_pix, a.n_grp, a.C, a.nsub, a.mw);
    int dev = 0, n_sm = 0;
    SPIIR_CUDA_TRY(cudaGetDevice(&dev));
    SPIIR_CUDA_TRY(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
    const int64_t ks = (int64_t)kTmRows * a.mw / a.nsub;  // samples of one template per item
    const int64_t items = (int64_t)((a.n_templates + a.nsub - 1) / a.nsub) * ((a.n + ks - 1) / ks);
    const int grid = (int)std::min<int64_t>(items, n_sm);
    if (a.mw == 16) {
        switch (a.nsub) {
            case 1: return launch_tmem_nsub<1, 16>(a, tab, grid, smem, stream);
            case 2: return launch_tmem_nsub<2, 16>(a, tab, grid, smem, stream);
            default: return launch_tmem_nsub<4, 16>(a, tab, grid, smem, stream);
        }
    }
    switch (a.nsub) {
        case 1: return launch_tmem_nsub<1, 8>(a, tab, grid, smem, stream);
        case 2: return launch_tmem_nsub<2, 8>(a, tab, grid, smem, stream);
        default: return launch_tmem_nsub<4, 8>(a, tab, grid, smem, stream);
    }
}

}  // namespace spiir
