// Signal-consistency statistic (Sec. II.C.2): for template t, detector I and sample k,
//     xi_I^2[k] = sum_{j=-Nj}^{Nj} |z_I[k + j] - z_I[k] A_t[j]|^2 / sum_{j=-Nj}^{Nj} (2 - 2 |A_t[j]|^2),
// A_t the template's autocorrelation, A[j] = R[j] / R[0], R[j] = sum_k conj(u[k]) u[k + j], and
// the network average xi_C^2 = (1 / N_d) sum_I xi_I^2 at the detectors' arrival times of the
// coherent argmax pixel.
//
// xi^2 kernel: a block covers 1024 samples of one (template, detector) with 128 threads of 8
// consecutive samples.  The SNR tile (1024 + 2 Nj + 8 samples) is staged in shared memory
// transposed by 8 (element x at (x % 8) L + x / 8), so the 32 threads of a warp reading sample
// 8 r + c hit 32 consecutive words.  Each thread keeps the 8-sample window z[k + j] of its
// samples in registers and slides it by one sample per tap (one shared load); the registers
// rotate with the tap index, unrolled by 8, so no moves are needed.  Per tap and sample the
// difference d = z[k + j] - z[k] A[j] and its squared modulus take three packed FP32 FMAs
// against a broadcast table entry (-A.re, -A.im, A.im, -A.re).
#include <algorithm>
#include <climits>

#include "coherent.cuh"

namespace spiir {

constexpr int kXiThreads = 128, kXiM = 8, kXiKT = kXiThreads * kXiM;
constexpr int kXiMaxLags = 1024;

__device__ __forceinline__ int xpos(int x, int L) { return (x & 7) * L + (x >> 3); }

// Plane stride of the transposed tile, a compile-time constant so that the 8 planes of the
// sliding-window reads sit at immediate offsets: at least (1024 + 2 Nj + 8) / 8 + 1, odd.
constexpr int xi_plane_stride(int n_lags) { return ((kXiKT + 2 * n_lags + kXiM) / 8 + 1) | 1; }
constexpr int kXiLSmall = xi_plane_stride(192), kXiLMax = xi_plane_stride(kXiMaxLags);

template <int L>
__global__ void __launch_bounds__(kXiThreads) k_xi2(const float2 *__restrict__ snr, int64_t pitch,
                                                    const float2 *__restrict__ A, int Nj, int64_t n, int n_det,
                                                    float *__restrict__ out, int64_t opitch) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int t = blockIdx.z, I = blockIdx.y, tid = threadIdx.x;
    const int64_t k0 = (int64_t)blockIdx.x * kXiKT;
    const int ntap = 2 * Nj + 1;
    const int W = kXiKT + 2 * Nj + kXiM;  // staged samples (W / 8 + 1 <= L, checked by the host)
    float4 *tab = reinterpret_cast<float4 *>(smem);           // [ntap]
    float2 *zt = reinterpret_cast<float2 *>(tab + ntap);      // [8 L] transposed tile
    __shared__ float den_part[kXiThreads / 32];
    const float2 *At = A + (int64_t)t * ntap;
    float dsum = 0.f;
    for (int j = tid; j < ntap; j += kXiThreads) {
        const float2 a = At[j];
        tab[j] = make_float4(-a.x, -a.y, a.y, -a.x);
        dsum += 2.f - 2.f * (a.x * a.x + a.y * a.y);
    }
    const float2 *row = snr + ((int64_t)t * n_det + I) * pitch + k0;
    const int64_t lim = n + 2 * Nj - k0;  // entries of the row this tile may read
    for (int x = tid; x < W; x += kXiThreads) zt[xpos(x, L)] = x < lim ? row[x] : make_float2(0.f, 0.f);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dsum += __shfl_xor_sync(0xffffffffu, dsum, o);
    if ((tid & 31) == 0) den_part[tid >> 5] = dsum;
    __syncthreads();
    float den = 0.f;
#pragma unroll
    for (int w = 0; w < kXiThreads / 32; ++w) den += den_part[w];

    const int base = kXiM * tid;  // tile position of this thread's first sample at tap -Nj
    if (k0 + base >= n) return;   // all of this thread's samples lie past the end (no barrier follows)
    u64 z0r[kXiM], z0i[kXiM], w[kXiM], acc[kXiM];
#pragma unroll
    for (int m = 0; m < kXiM; ++m) {
        const float2 c = zt[xpos(base + m + Nj, L)];
        z0r[m] = pack2(c.x, c.x);
        z0i[m] = pack2(c.y, c.y);
        const float2 v = zt[xpos(base + m, L)];
        w[m] = pack2(v.x, v.y);
        acc[m] = 0;
    }
    // tap s (j = s - Nj): logical window element m (sample m of this thread) is w[(m + s) % 8];
    // afterwards w[s % 8] takes the element that enters at the next tap, tile position
    // base + s + 8.  With s = 8 i + u that position lies in plane u at offset tid + i + 1, so
    // the 8 taps of a group read zg[u L] from one pointer with constant offsets.
    auto tap = [&](int s, int u, const float2 *zg) {
        const float4 e = tab[s];
        const u64 M1 = pack2(e.x, e.y), M2 = pack2(e.z, e.w);
#pragma unroll
        for (int m = 0; m < kXiM; ++m) {
            const u64 d = fma2(z0i[m], M2, fma2(z0r[m], M1, w[(m + u) & 7]));
            acc[m] = fma2(d, d, acc[m]);
        }
        const float2 v = zg[u * L];
        w[u] = pack2(v.x, v.y);
    };
    int s = 0;
    for (; s + 8 <= ntap; s += 8) {
        const float2 *zg = zt + tid + (s >> 3) + 1;
#pragma unroll
        for (int u = 0; u < 8; ++u) tap(s + u, u, zg);
    }
    {
        const float2 *zg = zt + tid + (s >> 3) + 1;
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (s + u < ntap) tap(s + u, u, zg);
    }

    float *orow = out + ((int64_t)t * n_det + I) * opitch + k0 + base;
    const float rden = 1.f / den;
    float r[kXiM];
#pragma unroll
    for (int m = 0; m < kXiM; ++m) {
        const float2 a = unpack2(acc[m]);
        r[m] = (a.x + a.y) * rden;
    }
    const int64_t kk = k0 + base;
#pragma unroll
    for (int m = 0; m < kXiM; ++m)
        if (kk + m < n) orow[m] = r[m];
}

// R[j] and R[0] of one template, one block per (lag, template)
__global__ void k_autocorr(const float2 *__restrict__ u, int64_t nr, int Nj, float2 *__restrict__ A) {
    const int j = blockIdx.x, t = blockIdx.y, tid = threadIdx.x, nt = blockDim.x;
    const float2 *ut = u + (int64_t)t * nr;
    float rj_x = 0.f, rj_y = 0.f, r0 = 0.f;
    for (int64_t k = tid; k < nr; k += nt) {
        const float2 a = ut[k];
        r0 = fmaf(a.x, a.x, fmaf(a.y, a.y, r0));
        if (k + j < nr) {
            const float2 b = ut[k + j];
            // conj(a) b
            rj_x = fmaf(a.x, b.x, fmaf(a.y, b.y, rj_x));
            rj_y = fmaf(a.x, b.y, fmaf(-a.y, b.x, rj_y));
        }
    }
    __shared__ float part[3][32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        rj_x += __shfl_xor_sync(0xffffffffu, rj_x, o);
        rj_y += __shfl_xor_sync(0xffffffffu, rj_y, o);
        r0 += __shfl_xor_sync(0xffffffffu, r0, o);
    }
    if ((tid & 31) == 0) {
        part[0][tid >> 5] = rj_x;
        part[1][tid >> 5] = rj_y;
        part[2][tid >> 5] = r0;
    }
    __syncthreads();
    if (tid == 0) {
        float sx = 0.f, sy = 0.f, s0 = 0.f;
        for (int w = 0; w < nt / 32; ++w) {
            sx += part[0][w];
            sy += part[1][w];
            s0 += part[2][w];
        }
        float2 *At = A + (int64_t)t * (2 * Nj + 1);
        At[Nj + j] = make_float2(sx / s0, sy / s0);
        At[Nj - j] = make_float2(sx / s0, -sy / s0);
    }
}

// xi_C^2 at every (template, sample): the mean of each detector's xi^2 at k + Delta_I(argmax)
__global__ void k_xi2_network(const float *__restrict__ xi, int64_t pitch, const int32_t *__restrict__ argmax,
                              const int16_t *__restrict__ dl, int n_det, int P, int H, int64_t Tn, int64_t n,
                              float *__restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= Tn) return;
    const int64_t t = i / n, k = i % n;
    const int p = argmax[i];
    if (p < 0 || p >= P) {
        out[i] = __int_as_float(0x7fc00000);  // NaN: not a pixel of this sky
        return;
    }
    float s = 0.f;
    for (int I = 0; I < n_det; ++I) s += xi[(t * n_det + I) * pitch + H + k + dl[p * n_det + I]];
    out[i] = s / n_det;
}

// xi^2 at candidate points (with the candidate scan of Sec. II.C.1 and the time shifts of
// Sec. II.C.3), in a persistent grid of warps.  With p the coherent argmax of a (candidate,
// shift) pair, detector J is read at x_J = e + Delta_J(p) - Delta_r(p) + shift_J (shift_J =
// -s c_J step for the c-th companion of the candidate's detector r); the lanes stride the taps
// j = -Nj .. Nj of each detector and the sums are reduced by shuffles.
struct XiPointArgs {
    const float2 *snr;  // [T][n_det][pitch], entry off + k is sample k
    int64_t pitch, off;
    int n_templates, n_det, n_pix;
    const float2 *A;  // [T][2 Nj + 1]
    int Nj;
    const int4 *cand;
    const int32_t *n_cand;
    int max_cand, first_shift, n_shifts;
    int64_t step;
    const int32_t *argmax;  // [max_cand][n_shifts]
    const int16_t *delays;  // [P][n_det]
    float *xi2;             // [max_cand][n_shifts]
    float *xi2_det;         // NULL or [max_cand][n_shifts][n_det]
};

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
    return v;
}

constexpr int kXiPtShifts = 8;  // shifts per warp item

// xi^2 of one detector row at sample x (entries x - Nj .. x + Nj), summed over the warp
__device__ __forceinline__ float xi_num(const float2 *__restrict__ row, const float2 *__restrict__ At, int Nj, int lane) {
    const float2 zc = row[Nj];
    float num = 0.f;
    for (int j = lane; j < 2 * Nj + 1; j += 32) {
        const float2 v = row[j], A = At[j];
        const float dr = v.x - (zc.x * A.x - zc.y * A.y);
        const float di = v.y - (zc.x * A.y + zc.y * A.x);
        num = fmaf(dr, dr, fmaf(di, di, num));
    }
    return warp_sum(num);
}

// One warp per (candidate, chunk of kXiPtShifts shifts).  The candidate's own detector r is
// read at its sample for every pixel and shift, so its xi^2 is evaluated once per item; the
// companions at each shift's argmax pixel.
__global__ void __launch_bounds__(256) k_xi2_points(const __grid_constant__ XiPointArgs a) {
    grid_dependency_wait();  // the argmax pixels and the candidates come from earlier kernels
    const int lane = threadIdx.x & 31;
    const int warps = gridDim.x * (blockDim.x >> 5);
    const int nc = min(*a.n_cand, a.max_cand);
    const int n_chunks = (a.n_shifts + kXiPtShifts - 1) / kXiPtShifts;
    const int64_t n_items = (int64_t)max(nc, 0) * n_chunks;
    const int ntap = 2 * a.Nj + 1;
    const float nan = __int_as_float(0x7fc00000);
    for (int64_t item = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); item < n_items; item += warps) {
        const int c = (int)(item / n_chunks), s0 = (int)(item % n_chunks) * kXiPtShifts;
        const int s1 = min(a.n_shifts, s0 + kXiPtShifts);
        const int4 cd = a.cand[c];
        const int r = cd.x, t = cd.y;
        const int64_t e = a.off + (int64_t)cd.z;
        const bool rec_ok = r >= 0 && r < a.n_det && t >= 0 && t < a.n_templates && cd.z >= 0 && e - a.Nj >= 0 &&
                            e + a.Nj < a.pitch;
        const float2 *At = a.A + (int64_t)(rec_ok ? t : 0) * ntap;
        // denominator sum_j (2 - 2 |A_t[j]|^2), shared by the detectors and shifts
        float den = 0.f;
        for (int j = lane; j < ntap; j += 32) {
            const float2 v = At[j];
            den += 2.f - 2.f * (v.x * v.x + v.y * v.y);
        }
        den = warp_sum(den);
        const float xi_r = rec_ok ? xi_num(a.snr + ((int64_t)t * a.n_det + r) * a.pitch + e - a.Nj, At, a.Nj, lane) / den
                                  : nan;
        for (int si = s0; si < s1; ++si) {
            const int64_t o = (int64_t)c * a.n_shifts + si;
            const int p = a.argmax[o];
            const int64_t s = (int64_t)a.first_shift + si;
            bool ok = rec_ok && p >= 0 && p < a.n_pix;
            float total = 0.f;
            int comp = 0;
            for (int J = 0; J < a.n_det && ok; ++J) {
                float xi;
                if (J == r) {
                    xi = xi_r;
                } else {
                    const int64_t x = e + a.delays[(int64_t)p * a.n_det + J] - a.delays[(int64_t)p * a.n_det + r] -
                                      s * (++comp) * a.step;
                    if (x - a.Nj < 0 || x + a.Nj >= a.pitch) {
                        ok = false;
                        break;
                    }
                    xi = xi_num(a.snr + ((int64_t)t * a.n_det + J) * a.pitch + x - a.Nj, At, a.Nj, lane) / den;
                }
                total += xi;
                if (a.xi2_det && lane == 0) a.xi2_det[o * a.n_det + J] = xi;
            }
            if (lane == 0) {
                a.xi2[o] = ok ? total / a.n_det : nan;
                if (!ok && a.xi2_det)
                    for (int J = 0; J < a.n_det; ++J) a.xi2_det[o * a.n_det + J] = nan;
            }
        }
    }
}

// xi^2 numerator of one detector row with the template's taps of this lane in registers: all
// NT loads of the row are issued at once (one memory round trip per row).  Taps past the last
// one are zero and add nothing.
template <int NT>
__device__ __forceinline__ float xi_num_reg(const float2 *__restrict__ row, const float2 (&Ar)[NT], int ntap, int Nj,
                                            int lane) {
    const float2 zc = row[Nj];
    float2 v[NT];
#pragma unroll
    for (int i = 0; i < NT; ++i) {
        const int j = lane + 32 * i;
        v[i] = j < ntap ? row[j] : make_float2(0.f, 0.f);
    }
    float num = 0.f;
#pragma unroll
    for (int i = 0; i < NT; ++i) {
        const float dr = v[i].x - (zc.x * Ar[i].x - zc.y * Ar[i].y);
        const float di = v[i].y - (zc.x * Ar[i].y + zc.y * Ar[i].x);
        num = fmaf(dr, dr, fmaf(di, di, num));
    }
    return warp_sum(num);
}

// The same statistic as k_xi2_points for templates of at most 32 NT taps and ND detectors, with
// the dependent loads batched: the template's taps and the denominator once per item, then lane
// i loads shift s0 + i's argmax pixel and that pixel's delays, which the shift loop takes by
// shuffles; the ND - 1 companion rows of a shift are loaded together (one memory round trip per
// shift).
template <int NT, int ND>
__global__ void __launch_bounds__(256) k_xi2_points_reg(const __grid_constant__ XiPointArgs a) {
    grid_dependency_wait();  // the argmax pixels and the candidates come from earlier kernels
    constexpr int NC = ND - 1;
    const int lane = threadIdx.x & 31;
    const int warps = gridDim.x * (blockDim.x >> 5);
    const int nc = min(*a.n_cand, a.max_cand);
    const int n_chunks = (a.n_shifts + kXiPtShifts - 1) / kXiPtShifts;
    const int64_t n_items = (int64_t)max(nc, 0) * n_chunks;
    const int ntap = 2 * a.Nj + 1;
    const float nan = __int_as_float(0x7fc00000);
    for (int64_t item = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); item < n_items; item += warps) {
        const int c = (int)(item / n_chunks), s0 = (int)(item % n_chunks) * kXiPtShifts;
        const int s1 = min(a.n_shifts, s0 + kXiPtShifts);
        const int4 cd = a.cand[c];
        const int r = cd.x, t = cd.y;
        const int64_t e = a.off + (int64_t)cd.z;
        const bool rec_ok = r >= 0 && r < ND && t >= 0 && t < a.n_templates && cd.z >= 0 && e - a.Nj >= 0 &&
                            e + a.Nj < a.pitch;
        const float2 *At = a.A + (int64_t)(rec_ok ? t : 0) * ntap;
        float2 Ar[NT];
        float den = 0.f;
#pragma unroll
        for (int i = 0; i < NT; ++i) {
            const int j = lane + 32 * i;
            Ar[i] = j < ntap ? At[j] : make_float2(0.f, 0.f);
            den += j < ntap ? 2.f - 2.f * (Ar[i].x * Ar[i].x + Ar[i].y * Ar[i].y) : 0.f;
        }
        den = warp_sum(den);
        // lane i: the argmax pixel of shift s0 + i and its delays
        int pl = -1, dl[ND];
#pragma unroll
        for (int J = 0; J < ND; ++J) dl[J] = 0;
        if (lane < s1 - s0) {
            pl = a.argmax[(int64_t)c * a.n_shifts + s0 + lane];
            if (pl >= 0 && pl < a.n_pix) {
#pragma unroll
                for (int J = 0; J < ND; ++J) dl[J] = a.delays[(int64_t)pl * ND + J];
            }
        }
        const float xi_r =
            rec_ok ? xi_num_reg<NT>(a.snr + ((int64_t)t * ND + r) * a.pitch + e - a.Nj, Ar, ntap, a.Nj, lane) / den : nan;
        for (int si = s0; si < s1; ++si) {
            const int64_t o = (int64_t)c * a.n_shifts + si;
            const int p = __shfl_sync(0xffffffffu, pl, si - s0);
            int dJ[ND], d_r = 0;
#pragma unroll
            for (int J = 0; J < ND; ++J) {
                dJ[J] = __shfl_sync(0xffffffffu, dl[J], si - s0);
                d_r = (J == r) ? dJ[J] : d_r;
            }
            const int64_t s = (int64_t)a.first_shift + si;
            bool ok = rec_ok && p >= 0 && p < a.n_pix;
            // companion q (detector order without r) of shift s reads around
            // e + Delta_J - Delta_r - s (q + 1) step
            const float2 *row[NC];
#pragma unroll
            for (int q = 0; q < NC; ++q) {
                int J = 0, dq = 0;
#pragma unroll
                for (int JJ = 0; JJ < ND; ++JJ)
                    if (JJ == (q < r ? q : q + 1)) {
                        J = JJ;
                        dq = dJ[JJ];
                    }
                const int64_t x = e + dq - d_r - s * (q + 1) * a.step;
                ok = ok && x - a.Nj >= 0 && x + a.Nj < a.pitch;
                row[q] = a.snr + ((int64_t)t * ND + J) * a.pitch + x - a.Nj;
            }
            if (!ok) {
                if (lane == 0) {
                    a.xi2[o] = nan;
                    if (a.xi2_det)
                        for (int J = 0; J < ND; ++J) a.xi2_det[o * ND + J] = nan;
                }
                continue;
            }
            float2 zc[NC], v[NC][NT];
#pragma unroll
            for (int q = 0; q < NC; ++q) {
                zc[q] = row[q][a.Nj];
#pragma unroll
                for (int i = 0; i < NT; ++i) {
                    const int j = lane + 32 * i;
                    v[q][i] = j < ntap ? row[q][j] : make_float2(0.f, 0.f);
                }
            }
            float xq[NC];
#pragma unroll
            for (int q = 0; q < NC; ++q) {
                float num = 0.f;
#pragma unroll
                for (int i = 0; i < NT; ++i) {
                    const float dr = v[q][i].x - (zc[q].x * Ar[i].x - zc[q].y * Ar[i].y);
                    const float di = v[q][i].y - (zc[q].x * Ar[i].y + zc[q].y * Ar[i].x);
                    num = fmaf(dr, dr, fmaf(di, di, num));
                }
                xq[q] = warp_sum(num) / den;
            }
            // the detectors' terms summed in detector order
            float total = 0.f;
#pragma unroll
            for (int J = 0; J < ND; ++J) {
                float xi = xi_r;
#pragma unroll
                for (int q = 0; q < NC; ++q)
                    if (J == (q < r ? q : q + 1)) xi = xq[q];
                total += xi;
                if (a.xi2_det && lane == 0) a.xi2_det[o * ND + J] = xi;
            }
            if (lane == 0) a.xi2[o] = total / ND;
        }
    }
}

template <int NT>
static int launch_xi2_nd(int nd, int grid, const XiPointArgs &a, cudaStream_t st) {
    auto kern = nd == 2 ? k_xi2_points_reg<NT, 2> : nd == 3 ? k_xi2_points_reg<NT, 3> : k_xi2_points_reg<NT, 4>;
    SPIIR_CUDA_TRY(launch_dependent(kern, dim3(grid), dim3(256), 0, st, a));
    return SPIIR_OK;
}

static int launch_xi2_reg(int NT, int nd, int grid, const XiPointArgs &a, cudaStream_t st) {
    switch (NT) {
        case 4: return launch_xi2_nd<4>(nd, grid, a, st);
        case 8: return launch_xi2_nd<8>(nd, grid, a, st);
        case 12: return launch_xi2_nd<12>(nd, grid, a, st);
        default: return launch_xi2_nd<16>(nd, grid, a, st);
    }
}

}  // namespace spiir

using namespace spiir;

extern "C" int spiir_xi2_candidates(spiir_sky_t sky, int T, const float *snr, int64_t pitch, int64_t off,
                                    const float *A, int n_lags, const int32_t *cand, const int32_t *n_cand,
                                    int max_cand, int first_shift, int n_shifts, int shift_step,
                                    const int32_t *argmax, float *xi2, float *xi2_det, void *stream) {
    clear_error();
    if (!sky) return fail(SPIIR_EINVAL, "sky is NULL");
    if (T < 1 || max_cand < 0 || n_shifts < 1 || first_shift < 0 || shift_step < 0 || off < 0 || pitch < 1)
        return fail(SPIIR_EINVAL, "n_templates = %d, max_cand = %d, first_shift = %d, n_shifts = %d, shift_step = %d",
                    T, max_cand, first_shift, n_shifts, shift_step);
    if (n_lags < 0 || n_lags > kXiMaxLags) return fail(SPIIR_EINVAL, "n_lags = %d outside [0, %d]", n_lags, kXiMaxLags);
    if ((int64_t)max_cand * n_shifts > INT_MAX) return fail(SPIIR_EINVAL, "max_cand x n_shifts above 2^31 - 1");
    if (!snr || !A || !n_cand || (max_cand > 0 && (!cand || !argmax || !xi2))) return fail(SPIIR_EINVAL, "NULL pointer");
    if (((uintptr_t)snr) % 8 || ((uintptr_t)A) % 8 || (cand && ((uintptr_t)cand) % 16))
        return fail(SPIIR_EINVAL, "snr and A must be 8-byte aligned, cand 16-byte aligned");
    if (max_cand == 0) return SPIIR_OK;
    XiPointArgs a{};
    a.snr = reinterpret_cast<const float2 *>(snr);
    a.pitch = pitch;
    a.off = off;
    a.n_templates = T;
    a.n_det = sky->n_det;
    a.n_pix = sky->n_pix;
    a.A = reinterpret_cast<const float2 *>(A);
    a.Nj = n_lags;
    a.cand = reinterpret_cast<const int4 *>(cand);
    a.n_cand = n_cand;
    a.max_cand = max_cand;
    a.first_shift = first_shift;
    a.n_shifts = n_shifts;
    a.step = shift_step;
    a.argmax = argmax;
    a.delays = sky->d_delays;
    a.xi2 = xi2;
    a.xi2_det = xi2_det;
    int dev = 0, n_sm = 0;
    SPIIR_CUDA_TRY(cudaGetDevice(&dev));
    SPIIR_CUDA_TRY(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
    const int64_t items = (int64_t)max_cand * ((n_shifts + kXiPtShifts - 1) / kXiPtShifts);
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((items + 7) / 8, (int64_t)n_sm * 8));
    const int nt = (2 * n_lags + 1 + 31) / 32;  // taps per lane
    const int nd = a.n_det;
    if (nd >= 2 && nd <= 4 && nt <= 16) {
        const int NT = nt <= 4 ? 4 : nt <= 8 ? 8 : nt <= 12 ? 12 : 16;
        SPIIR_TRY(launch_xi2_reg(NT, nd, grid, a, (cudaStream_t)stream));
    } else {
        SPIIR_CUDA_TRY(launch_dependent(k_xi2_points, dim3(grid), dim3(256), 0, (cudaStream_t)stream, a));
    }
    SPIIR_CUDA_TRY(cudaGetLastError());
    return SPIIR_OK;
}

extern "C" int spiir_autocorr(int T, const float *u, int64_t n_resp, int n_lags, float *A, void *stream) {
    clear_error();
    if (T < 1 || n_resp < 1) return fail(SPIIR_EINVAL, "n_templates = %d, n_resp = %lld", T, (long long)n_resp);
    if (n_lags < 0 || n_lags > kXiMaxLags) return fail(SPIIR_EINVAL, "n_lags = %d outside [0, %d]", n_lags, kXiMaxLags);
    if (!u || !A) return fail(SPIIR_EINVAL, "NULL pointer");
    k_autocorr<<<dim3((unsigned)(n_lags + 1), (unsigned)T), 256, 0, (cudaStream_t)stream>>>(
        reinterpret_cast<const float2 *>(u), n_resp, n_lags, reinterpret_cast<float2 *>(A));
    SPIIR_CUDA_TRY(cudaGetLastError());
    return SPIIR_OK;
}

extern "C" int spiir_xi2(int T, int n_det, const float *snr, int64_t snr_pitch, const float *A, int n_lags, int64_t n,
                         float *xi2, int64_t xi2_pitch, void *stream) {
    clear_error();
    if (T < 1 || n_det < 1 || n < 1) return fail(SPIIR_EINVAL, "n_templates = %d, n_det = %d, n = %lld", T, n_det, (long long)n);
    if (T > 65535 || n_det > 65535) return fail(SPIIR_EINVAL, "n_templates and n_det must be at most 65535");
    if (n_lags < 0 || n_lags > kXiMaxLags) return fail(SPIIR_EINVAL, "n_lags = %d outside [0, %d]", n_lags, kXiMaxLags);
    if (!snr || !A || !xi2) return fail(SPIIR_EINVAL, "NULL pointer");
    if (snr_pitch < n + 2 * (int64_t)n_lags)
        return fail(SPIIR_EINVAL, "snr_pitch %lld < n + 2 n_lags = %lld", (long long)snr_pitch,
                    (long long)(n + 2 * (int64_t)n_lags));
    if (xi2_pitch < n) return fail(SPIIR_EINVAL, "xi2_pitch %lld < n", (long long)xi2_pitch);
    if (((uintptr_t)snr) % 8 || ((uintptr_t)A) % 8) return fail(SPIIR_EINVAL, "snr and A must be 8-byte aligned");
    const int ntap = 2 * n_lags + 1;
    const int L = xi_plane_stride(n_lags) <= kXiLSmall ? kXiLSmall : kXiLMax;
    const size_t smem = (size_t)ntap * sizeof(float4) + (size_t)8 * L * sizeof(float2);
    SPIIR_TRY(set_max_dyn_smem((const void *)k_xi2<kXiLSmall>, 100 * 1024));
    SPIIR_TRY(set_max_dyn_smem((const void *)k_xi2<kXiLMax>, 100 * 1024));
    const dim3 grid((unsigned)((n + kXiKT - 1) / kXiKT), (unsigned)n_det, (unsigned)T);
    auto kern = L == kXiLSmall ? k_xi2<kXiLSmall> : k_xi2<kXiLMax>;
    kern<<<grid, kXiThreads, smem, (cudaStream_t)stream>>>(reinterpret_cast<const float2 *>(snr), snr_pitch,
                                                          reinterpret_cast<const float2 *>(A), n_lags, n, n_det, xi2,
                                                          xi2_pitch);
    SPIIR_CUDA_TRY(cudaGetLastError());
    return SPIIR_OK;
}

extern "C" int spiir_xi2_network(spiir_sky_t sky, int T, const float *xi2, int64_t xi2_pitch, const int32_t *argmax,
                                 int64_t n, float *out, void *stream) {
    clear_error();
    if (!sky) return fail(SPIIR_EINVAL, "sky is NULL");
    if (T < 1 || n < 1) return fail(SPIIR_EINVAL, "n_templates = %d, n = %lld", T, (long long)n);
    if (!xi2 || !argmax || !out) return fail(SPIIR_EINVAL, "NULL pointer");
    if (xi2_pitch < n + 2 * (int64_t)sky->halo)
        return fail(SPIIR_EINVAL, "xi2_pitch %lld < n + 2 H = %lld", (long long)xi2_pitch,
                    (long long)(n + 2 * (int64_t)sky->halo));
    const int64_t Tn = (int64_t)T * n;
    k_xi2_network<<<(unsigned)((Tn + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
        xi2, xi2_pitch, argmax, sky->d_delays, sky->n_det, sky->n_pix, sky->halo, Tn, n, out);
    SPIIR_CUDA_TRY(cudaGetLastError());
    return SPIIR_OK;
}
