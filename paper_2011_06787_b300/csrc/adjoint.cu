// Impulse response of a filter bank and its adjoint (reverse mode), for refining IIR
// coefficients against target templates.
//
// Forward (impulse mode), for every template t and filter l of t:
//     y_l[-1] = s_l,   y_l[k] = a1_l y_l[k-1] + b0_l [k == d_l],   u_t[k] = sum_l y_l[k]
// for k = 0 .. n-1 (Sec. II.B.1, Eq. (zk) driven by a unit impulse; the response is the
// commented closed form u(t) = sum_m b_m a_m^(t - t_m) plus the decay of the initial states).
//
// Reverse mode for a real loss L(u) with g = dL/dRe u + i dL/dIm u (PyTorch's convention,
// dL = Re sum conj(g) du):
//     lambda_l[n] = 0,   lambda_l[k] = g_t[k] + conj(a1_l) lambda_l[k+1]
//     dL/da1_l = sum_k lambda_l[k] conj(y_l[k-1]),   dL/db0_l = lambda_l[d_l] (d_l < n),
//     dL/ds_l  = conj(a1_l) lambda_l[0].
//
// Device mapping (K3): one block per template, one thread per filter.  The forward stores the
// state every C samples (C a multiple of 32).  The backward walks the C-sample segments in
// reverse: it recomputes the segment forward from its checkpoint keeping every 32nd state in
// shared memory, then for each 32-step block (in reverse) recomputes the 32 states into
// registers and runs the adjoint recurrence over them.  Each filter's gradient sums are
// blocked (32 steps, then a segment, then the total) to limit FP32 accumulation error.
// The per-template sum of the forward uses the same transposed shared-memory reduction as
// the filter bank.
#include <algorithm>

#include "common.cuh"

namespace spiir {

constexpr int kAdjR = 32;  // steps per reduction block / register block

__device__ __forceinline__ float2 cmul(float2 a, float2 y) {
    return make_float2(fmaf(a.x, y.x, -a.y * y.y), fmaf(a.x, y.y, a.y * y.x));
}

__global__ void k_impulse_fwd(const float2 *__restrict__ a1, const float2 *__restrict__ b0,
                              const int *__restrict__ dly, const float2 *__restrict__ s0, int F, int64_t n, int C,
                              float2 *__restrict__ u, float2 *__restrict__ ck, int nck) {
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int R = kAdjR;
    float2 *red = reinterpret_cast<float2 *>(smem);  // [blockDim][R + 1]
    const int t = blockIdx.x, l = threadIdx.x, nt = blockDim.x;
    const int warp = l >> 5, lane = l & 31, nw = nt >> 5;
    const bool act = l < F;
    const int64_t fi = (int64_t)t * F + l;
    const float2 a = act ? a1[fi] : make_float2(0.f, 0.f);
    const float2 b = act ? b0[fi] : make_float2(0.f, 0.f);
    const int64_t d = act ? dly[fi] : -1;
    float2 y = act ? s0[fi] : make_float2(0.f, 0.f);
    for (int64_t kb = 0; kb < n; kb += R) {
        const int nr = (int)min((int64_t)R, n - kb);
        if (ck && act && kb % C == 0) ck[fi * nck + kb / C] = y;  // y[kb - 1]
        for (int r = 0; r < nr; ++r) {
            y = cmul(a, y);
            if (kb + r == d) {
                y.x += b.x;
                y.y += b.y;
            }
            red[l * (R + 1) + r] = y;
        }
        __syncthreads();
        // each warp sums its 32 rows per column; lane r owns column r
        float2 acc = make_float2(0.f, 0.f);
        for (int i = 0; i < 32; ++i) {
            const float2 v = red[(warp * 32 + i) * (R + 1) + lane];
            acc.x += v.x;
            acc.y += v.y;
        }
        __syncthreads();
        red[warp * (R + 1) + lane] = acc;
        __syncthreads();
        if (l < nr) {
            float2 s = make_float2(0.f, 0.f);
            for (int w = 0; w < nw; ++w) {
                const float2 v = red[w * (R + 1) + l];
                s.x += v.x;
                s.y += v.y;
            }
            u[(int64_t)t * n + kb + l] = s;
        }
        __syncthreads();
    }
}

__global__ void k_impulse_bwd(const float2 *__restrict__ a1, const float2 *__restrict__ b0,
                              const int *__restrict__ dly, int F, int64_t n, int C, const float2 *__restrict__ ck,
                              int nck, const float2 *__restrict__ g, float2 *__restrict__ ga, float2 *__restrict__ gb,
                              float2 *__restrict__ gs) {
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int R = kAdjR;
    const int t = blockIdx.x, l = threadIdx.x, nt = blockDim.x;
    float2 *gsm = reinterpret_cast<float2 *>(smem);    // [C] gradient slice of this segment
    float2 *ick = gsm + C;                              // [C / R][nt] states at 32-step marks
    const bool act = l < F;
    const int64_t fi = (int64_t)t * F + l;
    const float2 a = act ? a1[fi] : make_float2(0.f, 0.f);
    const float2 b = act ? b0[fi] : make_float2(0.f, 0.f);
    const int64_t d = act ? dly[fi] : -1;
    const float2 ac = make_float2(a.x, -a.y);  // conj(a)
    float2 lam = make_float2(0.f, 0.f);
    float2 sa_tot = make_float2(0.f, 0.f), sb = make_float2(0.f, 0.f);
    const int nseg = (int)((n + C - 1) / C);
    for (int j = nseg - 1; j >= 0; --j) {
        const int64_t k0 = (int64_t)j * C;
        const int len = (int)min((int64_t)C, n - k0);
        __syncthreads();
        for (int i = l; i < len; i += nt) gsm[i] = g[(int64_t)t * n + k0 + i];
        // recompute the segment forward, keeping the state at every 32-step mark
        float2 y = act ? ck[fi * nck + j] : make_float2(0.f, 0.f);
        for (int i = 0; i < len; i += R) {
            ick[(i / R) * nt + l] = y;
            const int rl = min(R, len - i);
            for (int r = 0; r < rl; ++r) {
                y = cmul(a, y);
                if (k0 + i + r == d) {
                    y.x += b.x;
                    y.y += b.y;
                }
            }
        }
        __syncthreads();
        float2 sa_seg = make_float2(0.f, 0.f);
        for (int i = ((len - 1) / R) * R; i >= 0; i -= R) {
            const int rl = min(R, len - i);
            // yp[r] = y[k0 + i + r - 1], the previous state at step k0 + i + r
            float2 yp[R];
            float2 yy = ick[(i / R) * nt + l];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                yp[r] = yy;
                if (r < rl) {
                    yy = cmul(a, yy);
                    if (k0 + i + r == d) {
                        yy.x += b.x;
                        yy.y += b.y;
                    }
                }
            }
            float2 sa_blk = make_float2(0.f, 0.f);
#pragma unroll
            for (int r = R - 1; r >= 0; --r) {
                if (r < rl) {
                    const float2 gk = gsm[i + r];
                    // lambda = g + conj(a) lambda
                    const float lr = fmaf(ac.x, lam.x, fmaf(-ac.y, lam.y, gk.x));
                    const float li = fmaf(ac.x, lam.y, fmaf(ac.y, lam.x, gk.y));
                    lam = make_float2(lr, li);
                    // sum lambda conj(y_prev)
                    sa_blk.x = fmaf(lam.x, yp[r].x, fmaf(lam.y, yp[r].y, sa_blk.x));
                    sa_blk.y = fmaf(lam.y, yp[r].x, fmaf(-lam.x, yp[r].y, sa_blk.y));
                    if (k0 + i + r == d) sb = lam;
                }
            }
            sa_seg.x += sa_blk.x;
            sa_seg.y += sa_blk.y;
        }
        sa_tot.x += sa_seg.x;
        sa_tot.y += sa_seg.y;
    }
    if (act) {
        ga[fi] = sa_tot;
        gb[fi] = sb;
        gs[fi] = make_float2(fmaf(ac.x, lam.x, -ac.y * lam.y), fmaf(ac.x, lam.y, ac.y * lam.x));
    }
}

static int check_args(int T, int F, int64_t n, int C, int needs_ck) {
    if (T < 1 || F < 1 || F > 1024) return fail(SPIIR_EINVAL, "n_templates = %d, filters per template = %d (1..1024)", T, F);
    if (n < 1) return fail(SPIIR_EINVAL, "n = %lld < 1", (long long)n);
    if (needs_ck && (C < kAdjR || C % kAdjR != 0 || C > 8192))
        return fail(SPIIR_EINVAL, "ckpt_every = %d must be a multiple of %d in [%d, 8192]", C, kAdjR, kAdjR);
    return SPIIR_OK;
}

}  // namespace spiir

using namespace spiir;

extern "C" int spiir_impulse_forward(int T, int F, const float *a1, const float *b0, const int32_t *delay,
                                     const float *s0, int64_t n, float *u, int ckpt_every, float *ckpt, void *stream) {
    clear_error();
    SPIIR_TRY(check_args(T, F, n, ckpt_every, ckpt != nullptr));
    if (!a1 || !b0 || !delay || !s0 || !u) return fail(SPIIR_EINVAL, "NULL pointer");
    const int nt = (F + 31) / 32 * 32;
    const int C = ckpt ? ckpt_every : kAdjR;
    const int nck = (int)((n + C - 1) / C);
    const size_t smem = (size_t)nt * (kAdjR + 1) * sizeof(float2);
    static bool attr = false;
    if (!attr) {
        SPIIR_CUDA_TRY(cudaFuncSetAttribute(k_impulse_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
        attr = true;
    }
    k_impulse_fwd<<<T, nt, smem, (cudaStream_t)stream>>>(
        reinterpret_cast<const float2 *>(a1), reinterpret_cast<const float2 *>(b0), delay,
        reinterpret_cast<const float2 *>(s0), F, n, C, reinterpret_cast<float2 *>(u), reinterpret_cast<float2 *>(ckpt),
        nck);
    SPIIR_CUDA_TRY(cudaGetLastError());
    return SPIIR_OK;
}

extern "C" int spiir_impulse_backward(int T, int F, const float *a1, const float *b0, const int32_t *delay, int64_t n,
                                      const float *grad_u, int ckpt_every, const float *ckpt, float *grad_a1,
                                      float *grad_b0, float *grad_s0, void *stream) {
    clear_error();
    SPIIR_TRY(check_args(T, F, n, ckpt_every, 1));
    if (!a1 || !b0 || !delay || !grad_u || !ckpt || !grad_a1 || !grad_b0 || !grad_s0)
        return fail(SPIIR_EINVAL, "NULL pointer");
    const int nt = (F + 31) / 32 * 32;
    const int C = ckpt_every;
    const int nck = (int)((n + C - 1) / C);
    const size_t smem = (size_t)C * sizeof(float2) + (size_t)(C / kAdjR) * nt * sizeof(float2);
    if (smem > 227 * 1024) return fail(SPIIR_EUNSUPPORTED, "ckpt_every %d with %d filters needs %zu bytes of shared memory", C, F, smem);
    static bool attr = false;
    if (!attr) {
        SPIIR_CUDA_TRY(cudaFuncSetAttribute(k_impulse_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
        attr = true;
    }
    k_impulse_bwd<<<T, nt, smem, (cudaStream_t)stream>>>(
        reinterpret_cast<const float2 *>(a1), reinterpret_cast<const float2 *>(b0), delay, F, n, C,
        reinterpret_cast<const float2 *>(ckpt), nck, reinterpret_cast<const float2 *>(grad_u),
        reinterpret_cast<float2 *>(grad_a1), reinterpret_cast<float2 *>(grad_b0), reinterpret_cast<float2 *>(grad_s0));
    SPIIR_CUDA_TRY(cudaGetLastError());
    return SPIIR_OK;
}
