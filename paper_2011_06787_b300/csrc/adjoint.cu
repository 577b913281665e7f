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
// Device mapping (K3).  Both directions are parallel over checkpoint segments of C samples
// (C a multiple of 32):
//   forward   1. one thread per filter jumps from segment to segment in double-float (pairs
//                of FP32 numbers, about 44 significant bits),
//                y[(j+1)C - 1] = a^C y[jC - 1] + b a^((j+1)C - 1 - d) [jC <= d < (j+1)C],
//                and writes every segment's starting state (the checkpoints);
//             2. one block per (segment, template) runs the C steps in FP32 from its checkpoint,
//                two filters per packed pair and four per thread, and sums the template's
//                filters per sample with a transposed shared-memory reduction every 32 steps.
//   backward  1. per (segment, template, filter group): lambda over the segment in reverse from
//                a zero boundary (the segment's own contribution);
//             2. one thread per filter scans the segments in reverse in double-float: the boundary of
//                segment j is lambda at its end, lambda[jC] = local_j + conj(a)^len_j lambda_end;
//                grad_s0 = conj(a) lambda[0];
//             3. per (segment, template, filter group): states are recomputed from the
//                checkpoint (every 32nd kept in shared memory, each 32-step block recomputed
//                into registers), lambda runs in reverse from the boundary, and the segment's
//                share of grad_a1 (blocked sums) and grad_b0 (at k = d) are formed;
//             4. one thread per filter adds the segments' shares of grad_a1 in double-float, in order.
// The double-float jumps make every segment start exact to FP32 rounding, so FP32 error does not
// accumulate over the whole response.  Without a checkpoint buffer the forward runs one
// block per template sequentially over all n samples.
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
        if (ck && act && kb % C == 0) ck[(kb / C) * (int64_t)gridDim.x * F + fi] = y;  // y[kb - 1]
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

// Double-float arithmetic for the segment jumps: a value is the unevaluated sum hi + lo of two
// FP32 numbers (about 44 significant bits), built from the error-free transformations two-sum
// (Knuth) and two-product by FMA (Dekker's product with a fused multiply-add), as in the
// double-double library of Hida, Li and Bailey.  It runs on the FP32 pipe: no FP64 runs on the
// device.
struct df {
    float hi, lo;
};
__device__ __forceinline__ df two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ df quick_two_sum(float a, float b) {  // |a| >= |b|
    const float s = a + b;
    return {s, b - (s - a)};
}
__device__ __forceinline__ df df_add(df x, df y) {
    df s = two_sum(x.hi, y.hi);
    const df t = two_sum(x.lo, y.lo);
    s.lo += t.hi;
    s = quick_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return quick_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ df df_mul(df x, df y) {
    const float p = x.hi * y.hi;
    float e = fmaf(x.hi, y.hi, -p);
    e = fmaf(x.hi, y.lo, fmaf(x.lo, y.hi, e));
    return quick_two_sum(p, e);
}
__device__ __forceinline__ df df_neg(df x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ float df_round(df x) { return x.hi + x.lo; }

struct cdf {
    df x, y;
};
__device__ __forceinline__ cdf cdf_of(float2 v) { return {{v.x, 0.f}, {v.y, 0.f}}; }
__device__ __forceinline__ cdf cmul_df(cdf a, cdf b) {
    return {df_add(df_mul(a.x, b.x), df_neg(df_mul(a.y, b.y))), df_add(df_mul(a.x, b.y), df_mul(a.y, b.x))};
}
__device__ __forceinline__ cdf cadd_df(cdf a, cdf b) { return {df_add(a.x, b.x), df_add(a.y, b.y)}; }
__device__ __forceinline__ cdf cpow_df(cdf a, int64_t m) {
    cdf r{{1.f, 0.f}, {0.f, 0.f}};
    while (m > 0) {
        if (m & 1) r = cmul_df(r, a);
        a = cmul_df(a, a);
        m >>= 1;
    }
    return r;
}
__device__ __forceinline__ float2 f2(cdf a) { return make_float2(df_round(a.x), df_round(a.y)); }

// Forward 1: segment starting states (checkpoints) by double-float jumps.
__global__ void k_fwd_jump(const float2 *__restrict__ a1, const float2 *__restrict__ b0,
                           const int *__restrict__ dly, const float2 *__restrict__ s0, int64_t TF, int64_t n, int C,
                           int nck, float2 *__restrict__ ck) {
    const int64_t fi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (fi >= TF) return;
    const cdf a = cdf_of(a1[fi]), b = cdf_of(b0[fi]);
    const int64_t d = dly[fi];
    const cdf aC = cpow_df(a, C);
    cdf y = cdf_of(s0[fi]);
    ck[fi] = f2(y);
    for (int j = 0; j + 1 < nck; ++j) {
        const int64_t k0 = (int64_t)j * C;
        y = cmul_df(aC, y);
        if (d >= k0 && d < k0 + C) y = cadd_df(y, cmul_df(b, cpow_df(a, k0 + C - 1 - d)));
        ck[(int64_t)(j + 1) * TF + fi] = f2(y);
    }
}

constexpr int kFwdS = 4;  // filters per thread in the segment forward for templates above 320 filters
constexpr int kL1 = 64, kL2 = 16;  // mark spacings of the backward segment pass

// Forward 2: one block per (segment, template); u over the segment.
template <int S>
__global__ void __launch_bounds__(256) k_fwd_seg(const float2 *__restrict__ a1, const float2 *__restrict__ b0,
                                                 const int *__restrict__ dly, int F, int64_t n, int C, int nck,
                                                 const float2 *__restrict__ ck, float2 *__restrict__ u) {
    const int64_t TF = (int64_t)gridDim.y * F;
    constexpr int NP = S / 2, R = kAdjR;
    extern __shared__ __align__(16) unsigned char smem[];
    const int nt = blockDim.x, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nw = nt >> 5;
    float2 *red = reinterpret_cast<float2 *>(smem);  // [nt][R + 1]
    float2 *part = red + nt * (R + 1);               // [nw][R]
    const int t = blockIdx.y, j = blockIdx.x;
    const int64_t k0 = (int64_t)j * C;
    const int len = (int)min((int64_t)C, n - k0);
    u64 are[NP], aim[NP], naim[NP], yr[NP], yi[NP];
    float2 bv[S];
    int dd[S];
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        float2 a[2], y[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int s = 2 * p + h, f = tid * S + s;
            const bool ok = f < F;
            const int64_t fi = (int64_t)t * F + f;
            a[h] = ok ? a1[fi] : make_float2(0.f, 0.f);
            y[h] = ok ? ck[(int64_t)j * TF + fi] : make_float2(0.f, 0.f);
            bv[s] = ok ? b0[fi] : make_float2(0.f, 0.f);
            const int64_t e = ok ? (int64_t)dly[fi] - k0 : -1;
            dd[s] = (e >= 0 && e < len) ? (int)e : -1;  // step of the impulse inside this segment
        }
        are[p] = pack2(a[0].x, a[1].x);
        aim[p] = pack2(a[0].y, a[1].y);
        naim[p] = neg2(aim[p]);
        yr[p] = pack2(y[0].x, y[1].x);
        yi[p] = pack2(y[0].y, y[1].y);
    }
    float2 *row = red + tid * (R + 1);
    for (int kb = 0; kb < len; kb += R) {
        const int nr = min(R, len - kb);
        bool ev = false;
#pragma unroll
        for (int s = 0; s < S; ++s) ev |= dd[s] >= kb && dd[s] < kb + nr;
        // y = a y (+ b at k = d), then the thread's filters summed
        auto step = [&](int r, bool with_ev) {
            u64 accr = 0, acci = 0;
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                u64 nr_ = fma2(are[p], yr[p], mul2(naim[p], yi[p]));
                u64 ni_ = fma2(are[p], yi[p], mul2(aim[p], yr[p]));
                if (with_ev) {
                    float2 rr = unpack2(nr_), ii = unpack2(ni_);
                    if (dd[2 * p] == kb + r) {
                        rr.x += bv[2 * p].x;
                        ii.x += bv[2 * p].y;
                    }
                    if (dd[2 * p + 1] == kb + r) {
                        rr.y += bv[2 * p + 1].x;
                        ii.y += bv[2 * p + 1].y;
                    }
                    nr_ = pack2(rr.x, rr.y);
                    ni_ = pack2(ii.x, ii.y);
                }
                yr[p] = nr_;
                yi[p] = ni_;
                if (p == 0) {
                    accr = nr_;
                    acci = ni_;
                } else {
                    accr = add2(accr, nr_);
                    acci = add2(acci, ni_);
                }
            }
            const float2 ar = unpack2(accr), ai = unpack2(acci);
            row[r] = make_float2(ar.x + ar.y, ai.x + ai.y);
        };
        if (nr == R && !ev) {
#pragma unroll
            for (int r = 0; r < R; ++r) step(r, false);
        } else {
#pragma unroll 1
            for (int r = 0; r < nr; ++r) step(r, true);
        }
        __syncthreads();
        // each warp sums its 32 rows per column (lane r owns column r)
        {
            float2 acc = make_float2(0.f, 0.f);
#pragma unroll 8
            for (int i = 0; i < 32; ++i) {
                const float2 v = red[(warp * 32 + i) * (R + 1) + lane];
                acc.x += v.x;
                acc.y += v.y;
            }
            part[warp * R + lane] = acc;
        }
        __syncthreads();
        if (tid < nr) {
            float2 acc = make_float2(0.f, 0.f);
            for (int w = 0; w < nw; ++w) {
                const float2 v = part[w * R + tid];
                acc.x += v.x;
                acc.y += v.y;
            }
            u[(int64_t)t * n + k0 + kb + tid] = acc;
        }
        __syncthreads();
    }
}

// Backward 1: lambda over each segment in reverse from a zero boundary (one filter pair per
// thread); written to work[j][fi] (the workspace is segment-major, [nck + 2][T F]).
__global__ void k_bwd_local(const float2 *__restrict__ a1, int F, int64_t n, int C, int nck,
                            const float2 *__restrict__ g, float2 *__restrict__ work) {
    extern __shared__ __align__(16) unsigned char smem[];
    float4 *gq = reinterpret_cast<float4 *>(smem);  // [C] (g.re, g.re, g.im, g.im) of this segment
    const int t = blockIdx.y, j = blockIdx.x, nt = blockDim.x, tid = threadIdx.x;
    const int64_t k0 = (int64_t)j * C;
    const int len = (int)min((int64_t)C, n - k0);
    for (int i = tid; i < len; i += nt) {
        const float2 v = g[(int64_t)t * n + k0 + i];
        gq[i] = make_float4(v.x, v.x, v.y, v.y);
    }
    __syncthreads();
    const int f0 = 2 * (blockIdx.z * nt + tid);
    if (f0 >= F) return;
    const bool ok1 = f0 + 1 < F;
    const int64_t fi = (int64_t)t * F + f0;
    const float2 a0 = a1[fi], a1v = ok1 ? a1[fi + 1] : make_float2(0.f, 0.f);
    const u64 ar = pack2(a0.x, a1v.x), ai = pack2(a0.y, a1v.y), nai = neg2(ai);
    u64 lr = 0, li = 0;
    // lambda = g + conj(a) lambda:  re' = g.re + a.re l.re + a.im l.im,  im' = g.im + a.re l.im - a.im l.re
#pragma unroll 4
    for (int k = len - 1; k >= 0; --k) {
        const float4 gk = gq[k];
        const u64 nlr = fma2(ar, lr, fma2(ai, li, pack2(gk.x, gk.y)));
        const u64 nli = fma2(ar, li, fma2(nai, lr, pack2(gk.z, gk.w)));
        lr = nlr;
        li = nli;
    }
    const float2 r = unpack2(lr), i = unpack2(li);
    const int64_t TF = (int64_t)gridDim.y * F;
    work[j * TF + fi] = make_float2(r.x, i.x);
    if (ok1) work[j * TF + fi + 1] = make_float2(r.y, i.y);
}

// Backward 2: double-float reverse scan over the segments of one filter.  work[j][fi] holds the local
// lambda at the start of segment j on entry and lambda at its end (the boundary) on exit;
// work[nck][fi] and work[nck + 1][fi] receive a^16 and a^64 for the segment pass.
__global__ void k_bwd_scan(const float2 *__restrict__ a1, int64_t TF, int64_t n, int C, int nck,
                           float2 *__restrict__ work, float2 *__restrict__ gb, float2 *__restrict__ gs) {
    const int64_t fi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (fi >= TF) return;
    const cdf ac = cdf_of(make_float2(a1[fi].x, -a1[fi].y));  // conj(a)
    const cdf pC = cpow_df(ac, C), pL = cpow_df(ac, n - (int64_t)(nck - 1) * C);
    cdf lam{{0.f, 0.f}, {0.f, 0.f}};  // lambda at the end of the current segment (lambda[n] = 0)
    const cdf a = cdf_of(a1[fi]);
    work[(int64_t)nck * TF + fi] = f2(cpow_df(a, kL2));
    work[(int64_t)(nck + 1) * TF + fi] = f2(cpow_df(a, kL1));
    for (int j = nck - 1; j >= 0; --j) {
        float2 *w = work + (int64_t)j * TF + fi;
        const float2 loc = *w;
        *w = f2(lam);
        lam = cadd_df(cdf_of(loc), cmul_df(j == nck - 1 ? pL : pC, lam));
    }
    gs[fi] = f2(cmul_df(ac, lam));  // conj(a) lambda[0]
    gb[fi] = make_float2(0.f, 0.f);  // set by the segment holding d, if d < n
}

// Backward 3: per (segment, template, filter group), one filter pair per thread.  work[j][fi]:
// the boundary lambda on entry, the segment's share of grad_a1 on exit; work[nck][fi] and
// work[nck + 1][fi] hold a^16 and a^64 (double-float, rounded).  States at every 64th step come from
// jumps by a^64 (shared memory), at every 16th from jumps by a^16 (registers), and each 16-step
// block is recomputed step by step into registers before lambda runs back over it.
struct Pair {  // two filters as packed FP32 pairs: real parts, imaginary parts
    u64 re, im;
};
// y = m y for a packed complex pair m = (mr, mi), with nmi = -mi
__device__ __forceinline__ Pair pmul(u64 mr, u64 mi, u64 nmi, Pair y) {
    return {fma2(mr, y.re, mul2(nmi, y.im)), fma2(mr, y.im, mul2(mi, y.re))};
}

// One 16-step block of the segment pass, in reverse: states recomputed from the block's
// starting state into registers, then lambda = g + conj(a) lambda back over the block and the
// block's sum of lambda conj(y_prev).  CHECK: the slow form, for a block that is shorter than
// 16 steps or holds an impulse (ed: the impulse's step in the segment, or -1).
template <bool CHECK>
__device__ __forceinline__ void bwd_block(const float4 *gq, int s0i, int rl, Pair y, u64 ar, u64 ai, u64 nai,
                                          const float2 (&bv)[2], const int (&ed)[2], Pair &lam, u64 &bsr, u64 &bsi,
                                          float2 (&gbv)[2]) {
    Pair yp[kL2];
#pragma unroll
    for (int r = 0; r < kL2; ++r) {
        yp[r] = y;
        y = pmul(ar, ai, nai, y);
        if (CHECK) {
            float2 yr = unpack2(y.re), yi = unpack2(y.im);
            if (ed[0] == s0i + r) {
                yr.x += bv[0].x;
                yi.x += bv[0].y;
            }
            if (ed[1] == s0i + r) {
                yr.y += bv[1].x;
                yi.y += bv[1].y;
            }
            y = {pack2(yr.x, yr.y), pack2(yi.x, yi.y)};
        }
    }
#pragma unroll
    for (int r = kL2 - 1; r >= 0; --r) {
        if (CHECK && r >= rl) continue;
        const float4 gk = gq[s0i + r];
        const u64 nlr = fma2(ar, lam.re, fma2(ai, lam.im, pack2(gk.x, gk.y)));
        const u64 nli = fma2(ar, lam.im, fma2(nai, lam.re, pack2(gk.z, gk.w)));
        lam = {nlr, nli};
        bsr = fma2(nlr, yp[r].re, fma2(nli, yp[r].im, bsr));
        // - nlr y.im as a multiply-subtract, which the compiler folds into one packed FMA with a
        // negated product (an explicit sign flip would cost an integer operation per step)
        bsi = fma2(nli, yp[r].re, sub2(bsi, mul2(nlr, yp[r].im)));
        if (CHECK) {
            if (ed[0] == s0i + r) gbv[0] = make_float2(unpack2(nlr).x, unpack2(nli).x);
            if (ed[1] == s0i + r) gbv[1] = make_float2(unpack2(nlr).y, unpack2(nli).y);
        }
    }
}

__global__ void __launch_bounds__(256) k_bwd_seg(const float2 *__restrict__ a1, const float2 *__restrict__ b0,
                                                 const int *__restrict__ dly, int F, int64_t n, int C, int nck,
                                                 const float2 *__restrict__ ck, const float2 *__restrict__ g,
                                                 float2 *__restrict__ work, float2 *__restrict__ gb) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int t = blockIdx.y, j = blockIdx.x, nt = blockDim.x, tid = threadIdx.x;
    const int64_t TF = (int64_t)gridDim.y * F;
    float4 *gq = reinterpret_cast<float4 *>(smem);  // [C] (g.re, g.re, g.im, g.im)
    float4 *mk = gq + C;                             // [C / kL1][nt] states at 64-step marks (re pair, im pair)
    const int64_t k0 = (int64_t)j * C;
    const int len = (int)min((int64_t)C, n - k0);
    for (int i = tid; i < len; i += nt) {
        const float2 v = g[(int64_t)t * n + k0 + i];
        gq[i] = make_float4(v.x, v.x, v.y, v.y);
    }
    int f[2], ed[2];
    bool ok[2];
    float2 av[2], bv[2], y0[2], lam0[2], a16[2], a64[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        f[h] = 2 * (blockIdx.z * nt + tid) + h;
        ok[h] = f[h] < F;
        const int64_t fi = (int64_t)t * F + f[h];
        av[h] = ok[h] ? a1[fi] : make_float2(0.f, 0.f);
        bv[h] = ok[h] ? b0[fi] : make_float2(0.f, 0.f);
        y0[h] = ok[h] ? ck[(int64_t)j * TF + fi] : make_float2(0.f, 0.f);
        lam0[h] = ok[h] ? work[(int64_t)j * TF + fi] : make_float2(0.f, 0.f);
        a16[h] = ok[h] ? work[(int64_t)nck * TF + fi] : make_float2(0.f, 0.f);
        a64[h] = ok[h] ? work[(int64_t)(nck + 1) * TF + fi] : make_float2(0.f, 0.f);
        const int64_t e = ok[h] ? (int64_t)dly[fi] - k0 : -1;
        ed[h] = (e >= 0 && e < len) ? (int)e : -1;  // step of the impulse inside this segment
    }
    const u64 ar = pack2(av[0].x, av[1].x), ai = pack2(av[0].y, av[1].y), nai = neg2(ai);
    const u64 r16 = pack2(a16[0].x, a16[1].x), i16 = pack2(a16[0].y, a16[1].y), ni16 = neg2(i16);
    const u64 r64 = pack2(a64[0].x, a64[1].x), i64 = pack2(a64[0].y, a64[1].y), ni64 = neg2(i64);
    // impulse terms added by the jumps over the 64- and 16-step blocks that hold the impulse:
    // b a^(end - d), end the block's last step (double-float)
    float2 t64[2], t16[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        t64[h] = t16[h] = make_float2(0.f, 0.f);
        if (ed[h] >= 0) {
            const cdf a = cdf_of(av[h]), b = cdf_of(bv[h]);
            t64[h] = f2(cmul_df(b, cpow_df(a, kL1 - 1 - ed[h] % kL1)));
            t16[h] = f2(cmul_df(b, cpow_df(a, kL2 - 1 - ed[h] % kL2)));
        }
    }
    // 64-step marks
    const int nq = (len + kL1 - 1) / kL1;
    {
        Pair y{pack2(y0[0].x, y0[1].x), pack2(y0[0].y, y0[1].y)};
        for (int q = 0; q < nq; ++q) {
            mk[q * nt + tid] = make_float4(unpack2(y.re).x, unpack2(y.re).y, unpack2(y.im).x, unpack2(y.im).y);
            y = pmul(r64, i64, ni64, y);
            if ((ed[0] >= 0 && ed[0] / kL1 == q) || (ed[1] >= 0 && ed[1] / kL1 == q)) {
                float2 yr = unpack2(y.re), yi = unpack2(y.im);
                if (ed[0] >= 0 && ed[0] / kL1 == q) {
                    yr.x += t64[0].x;
                    yi.x += t64[0].y;
                }
                if (ed[1] >= 0 && ed[1] / kL1 == q) {
                    yr.y += t64[1].x;
                    yi.y += t64[1].y;
                }
                y = {pack2(yr.x, yr.y), pack2(yi.x, yi.y)};
            }
        }
    }
    __syncthreads();
    Pair lam{pack2(lam0[0].x, lam0[1].x), pack2(lam0[0].y, lam0[1].y)};
    u64 sar = 0, sai = 0;  // this segment's sum of lambda conj(y_prev)
    float2 gbv[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    for (int q = nq - 1; q >= 0; --q) {
        const int q0 = q * kL1, qlen = min(kL1, len - q0);
        // 16-step marks inside the 64-step block
        Pair sm[kL1 / kL2];
        {
            const float4 m = mk[q * nt + tid];
            Pair y{pack2(m.x, m.y), pack2(m.z, m.w)};
#pragma unroll
            for (int p = 0; p < kL1 / kL2; ++p) {
                sm[p] = y;
                y = pmul(r16, i16, ni16, y);
                const bool e0 = ed[0] >= q0 + p * kL2 && ed[0] < q0 + (p + 1) * kL2;
                const bool e1 = ed[1] >= q0 + p * kL2 && ed[1] < q0 + (p + 1) * kL2;
                if (e0 || e1) {
                    float2 yr = unpack2(y.re), yi = unpack2(y.im);
                    if (e0) {
                        yr.x += t16[0].x;
                        yi.x += t16[0].y;
                    }
                    if (e1) {
                        yr.y += t16[1].x;
                        yi.y += t16[1].y;
                    }
                    y = {pack2(yr.x, yr.y), pack2(yi.x, yi.y)};
                }
            }
        }
        u64 bsr = 0, bsi = 0;  // block sum
        const bool qev = (ed[0] >= q0 && ed[0] < q0 + kL1) || (ed[1] >= q0 && ed[1] < q0 + kL1);
        if (qlen == kL1 && !qev) {
#pragma unroll
            for (int p = kL1 / kL2 - 1; p >= 0; --p)
                bwd_block<false>(gq, q0 + p * kL2, kL2, sm[p], ar, ai, nai, bv, ed, lam, bsr, bsi, gbv);
        } else {
#pragma unroll
            for (int p = kL1 / kL2 - 1; p >= 0; --p)
                if (p * kL2 < qlen)
                    bwd_block<true>(gq, q0 + p * kL2, min(kL2, qlen - p * kL2), sm[p], ar, ai, nai, bv, ed, lam, bsr,
                                    bsi, gbv);
        }
        sar = add2(sar, bsr);
        sai = add2(sai, bsi);
    }
    const float2 sr = unpack2(sar), si = unpack2(sai);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        if (!ok[h]) continue;
        const int64_t fi = (int64_t)t * F + f[h];
        work[(int64_t)j * TF + fi] = make_float2(h ? sr.y : sr.x, h ? si.y : si.x);
        if (ed[h] >= 0) gb[fi] = gbv[h];
    }
}

// Backward 4: grad_a1 = the segments' shares added in double-float, in segment order.
__global__ void k_bwd_sum(int64_t TF, int nck, const float2 *__restrict__ work, float2 *__restrict__ ga) {
    const int64_t fi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (fi >= TF) return;
    df x{0.f, 0.f}, y{0.f, 0.f};
    for (int j = 0; j < nck; ++j) {
        const float2 v = work[(int64_t)j * TF + fi];
        x = df_add(x, {v.x, 0.f});
        y = df_add(y, {v.y, 0.f});
    }
    ga[fi] = make_float2(df_round(x), df_round(y));
}

// threads per block of the backward segment kernel (one filter pair each): groups of at most
// 256 pairs, as even as possible, within the shared-memory limit (g slice + 64-step marks)
static size_t bwd_seg_smem(int C, int nt) {
    return (size_t)C * sizeof(float4) + (size_t)((C + kL1 - 1) / kL1) * nt * sizeof(float4);
}
static int bwd_seg_threads(int F, int C) {
    const int pairs = (F + 1) / 2;
    for (int groups = (pairs + 255) / 256;; ++groups) {
        const int nt = ((pairs + groups - 1) / groups + 31) / 32 * 32;
        if (bwd_seg_smem(C, nt) <= 227 * 1024 || nt <= 32) return nt;
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
    cudaStream_t st = (cudaStream_t)stream;
    const auto A = reinterpret_cast<const float2 *>(a1);
    const auto B = reinterpret_cast<const float2 *>(b0);
    const auto S0 = reinterpret_cast<const float2 *>(s0);
    if (ckpt) {
        const int C = ckpt_every;
        const int nck = (int)((n + C - 1) / C);
        const int64_t TF = (int64_t)T * F;
        auto CK = reinterpret_cast<float2 *>(ckpt);
        k_fwd_jump<<<(unsigned)((TF + 127) / 128), 128, 0, st>>>(A, B, delay, S0, TF, n, C, nck, CK);
        SPIIR_CUDA_TRY(cudaGetLastError());
        // filters per thread: a template of up to 320 filters in one warp (S even, at most 10),
        // larger templates 4 per thread over several warps
        const int S = F <= 320 ? std::max(2, ((F + 31) / 32 + 1) / 2 * 2) : kFwdS;
        const int nt = ((F + S - 1) / S + 31) / 32 * 32;
        const size_t smem = (size_t)nt * (kAdjR + 1) * sizeof(float2) + (size_t)(nt / 32) * kAdjR * sizeof(float2);
        const dim3 grid((unsigned)nck, (unsigned)T);
        float2 *U = reinterpret_cast<float2 *>(u);
        // up to 256 threads x 33 float2 of reduction rows: above the 48 KB default
        SPIIR_TRY(set_max_dyn_smem((const void *)k_fwd_seg<2>, 100 * 1024));
        SPIIR_TRY(set_max_dyn_smem((const void *)k_fwd_seg<4>, 100 * 1024));
        SPIIR_TRY(set_max_dyn_smem((const void *)k_fwd_seg<6>, 100 * 1024));
        SPIIR_TRY(set_max_dyn_smem((const void *)k_fwd_seg<8>, 100 * 1024));
        SPIIR_TRY(set_max_dyn_smem((const void *)k_fwd_seg<10>, 100 * 1024));
        switch (S) {
            case 2: k_fwd_seg<2><<<grid, nt, smem, st>>>(A, B, delay, F, n, C, nck, CK, U); break;
            case 4: k_fwd_seg<4><<<grid, nt, smem, st>>>(A, B, delay, F, n, C, nck, CK, U); break;
            case 6: k_fwd_seg<6><<<grid, nt, smem, st>>>(A, B, delay, F, n, C, nck, CK, U); break;
            case 8: k_fwd_seg<8><<<grid, nt, smem, st>>>(A, B, delay, F, n, C, nck, CK, U); break;
            default: k_fwd_seg<10><<<grid, nt, smem, st>>>(A, B, delay, F, n, C, nck, CK, U); break;
        }
        SPIIR_CUDA_TRY(cudaGetLastError());
        return SPIIR_OK;
    }
    // no checkpoints: one block per template, sequential over all samples
    const int nt = (F + 31) / 32 * 32;
    const size_t smem = (size_t)nt * (kAdjR + 1) * sizeof(float2);
    if (smem > 227 * 1024)
        return fail(SPIIR_EUNSUPPORTED, "%d filters per template need a checkpoint buffer (the sequential form "
                                        "fits %d)", F, 227 * 1024 / ((kAdjR + 1) * (int)sizeof(float2)) / 32 * 32);
    SPIIR_TRY(set_max_dyn_smem((const void *)k_impulse_fwd, 227 * 1024));
    k_impulse_fwd<<<T, nt, smem, st>>>(A, B, delay, S0, F, n, kAdjR, reinterpret_cast<float2 *>(u), nullptr, 1);
    SPIIR_CUDA_TRY(cudaGetLastError());
    return SPIIR_OK;
}

extern "C" int spiir_impulse_backward(int T, int F, const float *a1, const float *b0, const int32_t *delay, int64_t n,
                                      const float *grad_u, int ckpt_every, const float *ckpt, float *grad_a1,
                                      float *grad_b0, float *grad_s0, float *workspace, void *stream) {
    clear_error();
    SPIIR_TRY(check_args(T, F, n, ckpt_every, 1));
    if (!a1 || !b0 || !delay || !grad_u || !ckpt || !grad_a1 || !grad_b0 || !grad_s0 || !workspace)
        return fail(SPIIR_EINVAL, "NULL pointer");
    const int C = ckpt_every;
    const int nck = (int)((n + C - 1) / C);
    const int64_t TF = (int64_t)T * F;
    const int nts = bwd_seg_threads(F, C);
    const size_t smem_seg = bwd_seg_smem(C, nts);
    if (smem_seg > 227 * 1024)
        return fail(SPIIR_EUNSUPPORTED, "ckpt_every %d needs %zu bytes of shared memory", C, smem_seg);
    cudaStream_t st = (cudaStream_t)stream;
    const auto A = reinterpret_cast<const float2 *>(a1);
    const auto B = reinterpret_cast<const float2 *>(b0);
    const auto G = reinterpret_cast<const float2 *>(grad_u);
    const auto CK = reinterpret_cast<const float2 *>(ckpt);
    auto W = reinterpret_cast<float2 *>(workspace);
    auto GA = reinterpret_cast<float2 *>(grad_a1);
    auto GB = reinterpret_cast<float2 *>(grad_b0);
    auto GS = reinterpret_cast<float2 *>(grad_s0);
    SPIIR_TRY(set_max_dyn_smem((const void *)k_bwd_local, 227 * 1024));
    SPIIR_TRY(set_max_dyn_smem((const void *)k_bwd_seg, 227 * 1024));
    const int ntl = 128;  // filter pairs per block of the local pass
    k_bwd_local<<<dim3((unsigned)nck, (unsigned)T, (unsigned)((F + 2 * ntl - 1) / (2 * ntl))), ntl,
                  (size_t)C * sizeof(float4), st>>>(A, F, n, C, nck, G, W);
    SPIIR_CUDA_TRY(cudaGetLastError());
    k_bwd_scan<<<(unsigned)((TF + 127) / 128), 128, 0, st>>>(A, TF, n, C, nck, W, GB, GS);
    SPIIR_CUDA_TRY(cudaGetLastError());
    k_bwd_seg<<<dim3((unsigned)nck, (unsigned)T, (unsigned)((F + 2 * nts - 1) / (2 * nts))), nts, smem_seg, st>>>(
        A, B, delay, F, n, C, nck, CK, G, W, GB);
    SPIIR_CUDA_TRY(cudaGetLastError());
    k_bwd_sum<<<(unsigned)((TF + 127) / 128), 128, 0, st>>>(TF, nck, W, GA);
    SPIIR_CUDA_TRY(cudaGetLastError());
    return SPIIR_OK;
}
