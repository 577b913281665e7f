// Single-detector candidate selection (Sec. II.C.1) and the coherent statistic evaluated at
// those candidates, at zero lag and under the time shifts of the background (Sec. II.C.3).
//
// Selection.  For every detector I and sample k the largest |z_I|^2 over the bank's templates
// (the lowest template among equals) is compared with threshold^2; a sample over it is a
// candidate of its template, and each (detector, template, second) keeps the largest one (the
// earliest among equals).  All decisions are taken on |z|^2 = re*re + im*im in FP32 with each
// operation rounded (no contraction), so that they are reproducible bit for bit.
//   k_select:  one warp per (32 samples, detector, 32 templates), lane = sample, coalesced
//              8-byte loads, 8 in flight per lane (one wave holds every task of a 1 s span of a
//              1024-template, 3-detector bank).  Each lane posts (|z|^2 bits, ~template) of
//              its best template to the sample's key with a 64-bit atomicMax: the largest
//              value wins, then the lowest template.
//   k_compact: launched as a programmatic dependent of k_select (scheduled while the selection
//              drains, it waits for its completion), one thread per key: a sample over the
//              threshold posts (|z|^2 bits, ~k) to its slot (detector, template, second) with a
//              64-bit atomicMax (the largest value, then the earliest sample); the last block
//              to finish walks the slots in order and writes a record per occupied slot with a
//              block-wide prefix sum.  Keys, slots and the block counter are cleared on the way,
//              so the workspace is zero again for the next call; the count stays on the device.
//
// Candidate-driven scan.  A candidate (detector r, template t, sample k) is evaluated at every
// pixel p with detector r read at its own sample and each other detector J at
// k + Delta_J(p) - Delta_r(p) + shift_J, shift_J = -s c_J step for time shift s (c_J = 1, 2, ...
// the companions of r in detector order; s = 0 is the foreground).
//   k_points_chunked (skies whose windows fit 192 samples): one block per (candidate, chunk of
//              16 shifts, or 1 at zero lag, 8 for four detectors) in a persistent grid.  The
//              companions' windows of the chunk's shifts sit in shared memory, and the next
//              item's windows are copied (cp.async) while the current one is evaluated; the
//              reference detector's term is formed once per pixel; the lanes keep a maximum per
//              shift, reduced over the warp by two redux.sync per shift (the largest value, then
//              the lowest pixel holding it) and over the block through shared memory.
//   k_points:  the general form, one block per (candidate, shift), for wide windows or large
//              tables.
// Both keep the largest statistic (the lowest pixel among equals) and the null stream at that
// pixel, with the arithmetic of the all-sky scan.
#include <algorithm>
#include <climits>
#include <cmath>
#include <type_traits>
#include <vector>

#include "coherent.cuh"

namespace spiir {

constexpr int kSelBlock = 256;    // 8 warps, one task each
constexpr int kSelTaskT = 32;     // templates per warp task
constexpr int kSelUnroll = 8;     // loads in flight per lane
constexpr int kCompThreads = 1024;
constexpr int kCompSlots = 4;     // consecutive slots per thread and round
constexpr int kPtThreads = 256;
constexpr int kPtMaxSmem = 200 * 1024;
constexpr int kPtChunkSmem = 110 * 1024;  // two blocks per SM

__device__ __forceinline__ u64 lds64(const float *p) { return *reinterpret_cast<const u64 *>(p); }

__device__ __forceinline__ float mag2_rn(float2 z) { return __fadd_rn(__fmul_rn(z.x, z.x), __fmul_rn(z.y, z.y)); }

// Task = (detector I, column of 32 samples, chunk of kSelTaskT templates), one per warp, lane =
// sample.
__global__ void __launch_bounds__(kSelBlock) k_select(const float2 *__restrict__ snr, int64_t pitch, int64_t off,
                                                     int T, int n_det, int n, int n_cols, int n_chunks,
                                                     u64 *__restrict__ keys) {
    grid_dependents_trigger();  // the compaction grid may be scheduled now
    const int lane = threadIdx.x & 31;
    const int task = blockIdx.x * (kSelBlock / 32) + (threadIdx.x >> 5);
    if (task >= n_cols * n_det * n_chunks) return;
    const int col = task % n_cols, rest = task / n_cols;
    const int I = rest % n_det;
    const int t0 = (rest / n_det) * kSelTaskT, t1 = min(T, t0 + kSelTaskT);
    const int k = col * 32 + lane;
    if (k >= n) return;
    const int64_t ts = (int64_t)n_det * pitch;  // template stride
    const float2 *p = snr + ((int64_t)t0 * n_det + I) * pitch + off + k;
    float best = -1.f;
    int bt = INT_MAX;
    int t = t0;
    for (; t + kSelUnroll <= t1; t += kSelUnroll, p += kSelUnroll * ts) {
        float2 v[kSelUnroll];
#pragma unroll
        for (int j = 0; j < kSelUnroll; ++j) v[j] = p[j * ts];
#pragma unroll
        for (int j = 0; j < kSelUnroll; ++j) {
            const float m = mag2_rn(v[j]);
            if (m > best) {
                best = m;
                bt = t + j;
            }
        }
    }
    for (; t < t1; ++t, p += ts) {
        const float m = mag2_rn(*p);
        if (m > best) {
            best = m;
            bt = t;
        }
    }
    if (bt != INT_MAX)
        atomicMax(keys + (int64_t)I * n + k, ((u64)__float_as_uint(best) << 32) | (u64)(0xFFFFFFFFu - (uint32_t)bt));
}

// Exclusive prefix sum over the block of one int per thread (blockDim.x = kCompThreads); the
// total in *total.  Ends with the block synchronised.
__device__ __forceinline__ int block_exclusive_sum(int v, int *s_warp, int *total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) s_warp[w] = x;
    __syncthreads();
    if (w == 0) {
        const int wv = s_warp[lane];
        int wx = wv;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, wx, d);
            if (lane >= d) wx += y;
        }
        s_warp[lane] = wx - wv;
        if (lane == 31) *total = wx;
    }
    __syncthreads();
    const int r = s_warp[w] + x - v;
    __syncthreads();  // s_warp and total may be reused
    return r;
}

// Launched as a programmatic dependent of k_select, one thread per key.  Index arithmetic in 32
// bits: the host checks that n_det n and n_det T n_sec are below 2^31.
//  1. every sample over the threshold posts (|z|^2 bits, ~k) of its best template to the slot
//     (detector, template, second) with a 64-bit atomicMax (the largest value, then the
//     earliest sample); keys are cleared;
//  2. the last block to finish 1 (a counter; each block fences its slot updates before
//     counting) writes one record per occupied slot in (detector, template, second) order,
//     thread i taking kCompSlots consecutive slots of each round, and clears the slots and the
//     counter.
__global__ void __launch_bounds__(kCompThreads) k_compact(u64 *__restrict__ keys, int n, int n_det, int T,
                                                         float thr2, int per_second, u64 *__restrict__ slots,
                                                         int n_sec, unsigned *__restrict__ done,
                                                         int4 *__restrict__ cand, int max_cand,
                                                         int32_t *__restrict__ n_cand) {
    __shared__ int s_warp[32];
    __shared__ int s_total;
    __shared__ bool s_last;
    grid_dependency_wait();  // k_select's keys are complete and visible after this
    const int i = blockIdx.x * kCompThreads + (int)threadIdx.x;
    if (i < n_det * n) {
        const u64 kv = __ldcg(reinterpret_cast<const unsigned long long *>(keys + i));
        if (kv) {
            keys[i] = 0;
            if (__uint_as_float((uint32_t)(kv >> 32)) > thr2) {
                const int I = i / n, k = i - I * n;
                const int t = (int)(0xFFFFFFFFu - (uint32_t)kv);
                atomicMax(slots + ((I * T + t) * n_sec + k / per_second),
                          (kv & 0xFFFFFFFF00000000ull) | (u64)(0xFFFFFFFFu - (uint32_t)k));
            }
        }
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const int n_slots = n_det * T * n_sec;
    int64_t base = 0;
    for (int c0 = 0; c0 < n_slots; c0 += kCompThreads * kCompSlots) {
        const int s0 = c0 + (int)threadIdx.x * kCompSlots;
        u64 sv[kCompSlots];
        int cnt = 0;
#pragma unroll
        for (int j = 0; j < kCompSlots; ++j) {
            sv[j] = s0 + j < n_slots ? __ldcg(reinterpret_cast<const unsigned long long *>(slots + s0 + j)) : 0ull;
            cnt += sv[j] != 0;
        }
        int64_t pos = base + block_exclusive_sum(cnt, s_warp, &s_total);
#pragma unroll
        for (int j = 0; j < kCompSlots; ++j) {
            if (!sv[j]) continue;
            slots[s0 + j] = 0;
            if (pos < max_cand) {
                const int it = n_sec == 1 ? s0 + j : (s0 + j) / n_sec;  // I * T + t
                const int I = it / T;
                cand[pos] = make_int4(I, it - I * T, (int)(0xFFFFFFFFu - (uint32_t)sv[j]), (int)(sv[j] >> 32));
            }
            ++pos;
        }
        base += s_total;
    }
    if (threadIdx.x == 0) {
        *n_cand = (int32_t)std::min<int64_t>(base, INT_MAX);
        *done = 0;
    }
}

struct PointArgs {
    const float2 *snr;  // [T][n_det][pitch], entry off + k is sample k
    int64_t pitch, off;
    int n_templates;
    const int4 *cand;  // [max_cand] (detector, template, sample, |z|^2 bits)
    const int32_t *n_cand;
    int max_cand;
    int first_shift, n_shifts;
    int64_t step;
    const void *table;  // TabEntry<ND>[n_pix]
    const float *u_null;
    int n_pix, H;
    int dmin[4][4], dmax[4][4];  // range of Delta_J - Delta_r over the sky, [r][J]
    int Wmax;                    // largest window, entries per detector in shared memory
    size_t tab_bytes;            // table staged in shared memory (0: read from global)
    const void *ptab;            // PtEnt<ND>[ND][n_pix]: per-reference entries of the chunked scan
    float *max_stat;             // [max_cand][n_shifts]
    int32_t *argmax;
    float *null_stat;
};

struct Best {
    float v;
    int p;
    float nul;
};
__device__ __forceinline__ void take(Best &a, float v, int p, float nul) {
    if (v > a.v || (v == a.v && p < a.p)) {
        a.v = v;
        a.p = p;
        a.nul = nul;
    }
}

template <int ND, bool SMEM_TAB>
__global__ void __launch_bounds__(kPtThreads) k_points(const __grid_constant__ PointArgs a) {
    grid_dependency_wait();  // the candidate records and count come from the previous kernel
    using Entry = TabEntry<ND>;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ Best s_red[kPtThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const Entry *tab = reinterpret_cast<const Entry *>(a.table);
    if (SMEM_TAB) {
        const uint4 *src = reinterpret_cast<const uint4 *>(a.table);
        uint4 *dst = reinterpret_cast<uint4 *>(smem);
        for (size_t i = tid; i < a.tab_bytes / 16; i += kPtThreads) dst[i] = src[i];
        tab = reinterpret_cast<const Entry *>(smem);
    }
    float2 *win = reinterpret_cast<float2 *>(smem + a.tab_bytes);  // [ND][Wmax]
    const int nc = min(*a.n_cand, a.max_cand);
    const int64_t n_items = (int64_t)max(nc, 0) * a.n_shifts;
    for (int64_t item = blockIdx.x; item < n_items; item += gridDim.x) {
        const int c = (int)(item / a.n_shifts);
        const int si = (int)(item % a.n_shifts);
        const int4 cd = a.cand[c];
        const int r = cd.x, t = cd.y;
        const int64_t e = a.off + (int64_t)cd.z;
        const int64_t s = (int64_t)a.first_shift + si;
        const int64_t o = (int64_t)c * a.n_shifts + si;
        // the first entry of each detector's window; the item is void if any read leaves the row
        bool ok = r >= 0 && r < ND && t >= 0 && t < a.n_templates && cd.z >= 0;
        int64_t lo[ND];
        int len[ND];
        if (ok) {
            int comp = 0;
#pragma unroll
            for (int J = 0; J < ND; ++J) {
                const int64_t sh = (J == r) ? 0 : -s * (++comp) * a.step;
                lo[J] = e + sh + a.dmin[r][J];
                len[J] = a.dmax[r][J] - a.dmin[r][J] + 1;
                ok = ok && lo[J] >= 0 && lo[J] + len[J] <= a.pitch;
            }
        }
        if (!ok) {
            if (tid == 0) {
                a.max_stat[o] = __int_as_float(0x7fc00000);
                a.argmax[o] = -1;
                a.null_stat[o] = __int_as_float(0x7fc00000);
            }
            continue;
        }
        __syncthreads();  // the previous item is done with the windows (and the table is staged)
#pragma unroll
        for (int J = 0; J < ND; ++J) {
            const float2 *row = a.snr + ((int64_t)t * ND + J) * a.pitch + lo[J];
            for (int j = tid; j < len[J]; j += kPtThreads) win[J * a.Wmax + j] = row[j];
        }
        __syncthreads();
        int base[ND];  // window index of pixel p for detector J: off[J] - off[r] - dmin[r][J]
#pragma unroll
        for (int J = 0; J < ND; ++J) base[J] = J * a.Wmax - a.dmin[r][J];
        Best b{-1.f, INT_MAX, 0.f};
        for (int p = tid; p < a.n_pix; p += kPtThreads) {
            const Entry en = tab[p];
            int orr = 0;  // off[r], selected without indexing the entry at run time
#pragma unroll
            for (int J = 0; J < ND; ++J) orr = (J == r) ? en.off[J] : orr;
            float y0r = 0.f, y0i = 0.f, y1r = 0.f, y1i = 0.f;
#pragma unroll
            for (int J = 0; J < ND; ++J) {
                const float2 wv = win[base[J] + en.off[J] - orr];
                y0r = fmaf(en.u[J][0], wv.x, y0r);
                y0i = fmaf(en.u[J][0], wv.y, y0i);
                y1r = fmaf(en.u[J][1], wv.x, y1r);
                y1i = fmaf(en.u[J][1], wv.y, y1i);
            }
            const float v = fmaf(y1i, y1i, fmaf(y1r, y1r, fmaf(y0i, y0i, y0r * y0r)));
            if (v > b.v) {
                b.v = v;
                b.p = p;
            }
        }
        if (ND > 2 && b.p != INT_MAX) {
            const Entry en = tab[b.p];
            int orr = 0;
#pragma unroll
            for (int J = 0; J < ND; ++J) orr = (J == r) ? en.off[J] : orr;
            const float *un = a.u_null + (int64_t)b.p * ND * (ND - 2);
            float nul = 0.f;
            for (int j = 0; j < ND - 2; ++j) {
                float cr = 0.f, ci = 0.f;
#pragma unroll
                for (int J = 0; J < ND; ++J) {
                    const float2 wv = win[base[J] + en.off[J] - orr];
                    const float u = un[J * (ND - 2) + j];
                    cr = fmaf(u, wv.x, cr);
                    ci = fmaf(u, wv.y, ci);
                }
                nul = fmaf(cr, cr, fmaf(ci, ci, nul));
            }
            b.nul = nul;
        }
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            const float v = __shfl_down_sync(0xffffffffu, b.v, d);
            const int p = __shfl_down_sync(0xffffffffu, b.p, d);
            const float nl = __shfl_down_sync(0xffffffffu, b.nul, d);
            take(b, v, p, nl);
        }
        if (lane == 0) s_red[wid] = b;
        __syncthreads();
        if (tid == 0) {
            for (int q = 1; q < kPtThreads / 32; ++q) take(b, s_red[q].v, s_red[q].p, s_red[q].nul);
            const bool found = b.p != INT_MAX;
            a.max_stat[o] = found ? b.v : __int_as_float(0x7fc00000);
            a.argmax[o] = found ? b.p : -1;
            a.null_stat[o] = found ? b.nul : __int_as_float(0x7fc00000);
        }
    }
}

// ---------------------------------------------------------------------------------------
// Chunked candidate scan: one block per (candidate, chunk of S consecutive shifts), for skies
// whose windows (the range of Delta_J - Delta_r) fit in kPtWP entries and whose table fits in
// shared memory with the windows of S shifts.
//
// The reference detector is never shifted, so its term U_s[p][r] w_r is the same for every
// shift and is formed once per pixel; each shift adds the N_d - 1 companion terms.  The
// windows are laid out [shift][companion][kPtWP], so that for one pixel the address of every
// shift differs by a compile-time constant.  Each thread keeps a running maximum per shift;
// a warp reduces each shift's (value, pixel) pairs with two integer reductions (redux.sync on
// the value bits, which order as unsigned integers because the statistic is >= 0, then on the
// pixels that hold the maximum), then the warps combine through shared memory.
constexpr int kPtWP = 192;        // window entries per (shift, companion): wide skies
constexpr int kPtWPNarrow = 96;   // the same when the relative delays span at most 96 samples
constexpr int kPtChunkThreads = 128;

__device__ __forceinline__ void take_pair(float &kv, int &kp, float rv, int rp) {
    if (rv > kv || (rv == kv && rp < kp)) {
        kv = rv;
        kp = rp;
    }
}

__device__ __forceinline__ void cp_async8(void *dst_smem, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst_smem)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Per-reference-detector entry of the chunked scan: for reference detector r and pixel p, the
// signal columns U_s[p][r] and U_s[p][J_q] of its companions J_q (q = 0 .. N_d - 2, detector
// order without r), each companion's window index Delta_Jq(p) - Delta_r(p) - min over the sky of
// the same difference (10 bits each, packed), and p.  Two or three 16-byte loads per pixel
// replace the gather of the general entry's fields at run-time detector indices.
// Order: the sky in chunks of kPtChunkThreads consecutive pixels, each chunk arranged by
// order_chunk so that the 16 lanes of a half-warp read window entries in distinct bank pairs as
// far as the sky allows (fewer shared-memory bank conflicts), while every thread still visits
// its pixels in increasing p (one per chunk), which keeps the lowest pixel among equal
// statistics with a plain comparison.
template <int ND>
struct __align__(16) PtEnt {
    float ur[2];
    float uq[ND - 1][2];
    uint32_t idx;   // idx_q = (idx >> 10 q) & 1023
    int p;          // pixel index
};

// One (candidate, chunk) work item as every thread of the block sees it.
template <int ND>
struct PtItem {
    int c, s_first, ns, r, t;
    int64_t e;
    uint32_t okmask;  // bit i: every read of shift column i stays inside the row
    int Jq[ND - 1], dmn[ND - 1], dmx[ND - 1];
};

// Items number fewer than 2^30 (the host checks), so their arithmetic is 32-bit.
template <int ND, int S>
__device__ __forceinline__ PtItem<ND> decode_item(const PointArgs &a, int item, int n_chunks, int lane) {
    constexpr int NC = ND - 1;
    PtItem<ND> it;
    it.c = item / n_chunks;
    it.s_first = (item - it.c * n_chunks) * S;
    it.ns = min(S, a.n_shifts - it.s_first);
    const int4 cd = a.cand[it.c];
    it.r = cd.x;
    it.t = cd.y;
    it.e = a.off + (int64_t)cd.z;
    const bool rec_ok = it.r >= 0 && it.r < ND && it.t >= 0 && it.t < a.n_templates && cd.z >= 0 && it.e < a.pitch;
#pragma unroll
    for (int q = 0; q < NC; ++q) {
        it.Jq[q] = (q < it.r) ? q : q + 1;
        it.dmn[q] = rec_ok ? a.dmin[it.r][it.Jq[q]] : 0;
        it.dmx[q] = rec_ok ? a.dmax[it.r][it.Jq[q]] : 0;
    }
    // lane i tests shift column i; companion q of shift s reads entries
    // e - s (q + 1) step + [dmn[q], dmx[q]]
    bool ok = rec_ok && lane < it.ns;
    if (ok) {
        const int64_t s = (int64_t)a.first_shift + it.s_first + lane;
#pragma unroll
        for (int q = 0; q < NC; ++q) {
            const int64_t x = it.e - s * (q + 1) * a.step;
            ok = ok && x + it.dmn[q] >= 0 && x + it.dmx[q] < a.pitch;
        }
    }
    it.okmask = __ballot_sync(0xffffffffu, ok);
    return it;
}

// Start the copies of an item's windows into buf ([S][NC][WP]): warp w copies shift columns
// w, w + 4, ... of each companion, lanes striding a window with 8-byte asynchronous copies.  A
// companion's windows all have the same length and lie (q + 1) step samples apart per column, so
// the source offset is stepped rather than recomputed.
template <int ND, int S, int WP>
__device__ __forceinline__ void stage_item(const PointArgs &a, const PtItem<ND> &it, float2 *buf, int wid, int lane) {
    constexpr int NC = ND - 1;
    constexpr int kWarps = kPtChunkThreads / 32;
#pragma unroll
    for (int q = 0; q < NC; ++q) {
        const int len = it.dmx[q] - it.dmn[q] + 1;
        const int64_t s0 = (int64_t)a.first_shift + it.s_first + wid;
        int64_t o = ((int64_t)it.t * ND + it.Jq[q]) * a.pitch + it.e - s0 * (q + 1) * a.step + it.dmn[q];
        const int64_t o_step = (int64_t)kWarps * (q + 1) * a.step;
        float2 *dst = buf + (wid * NC + q) * WP;
        for (int i = wid; i < S; i += kWarps, o -= o_step, dst += kWarps * NC * WP) {
            if (!((it.okmask >> i) & 1u)) continue;
            const float2 *row = a.snr + o;
            for (int j = lane; j < len; j += 32) cp_async8(dst + j, row + j);
        }
    }
}

template <int ND, int S, int WP>
__global__ void __launch_bounds__(kPtChunkThreads, 4) k_points_chunked(const __grid_constant__ PointArgs a) {
    grid_dependency_wait();  // the candidate records and count come from the previous kernel
    using Entry = TabEntry<ND>;
    constexpr int NC = ND - 1;                    // companions of the reference detector
    constexpr int kShiftWords = NC * WP;          // float2 entries per shift
    constexpr int kWarps = kPtChunkThreads / 32;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ float s_v[kWarps][S];
    __shared__ int s_p[kWarps][S];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const Entry *__restrict__ tab = reinterpret_cast<const Entry *>(a.table);  // read through L1
    const PtEnt<ND> *__restrict__ ptab = reinterpret_cast<const PtEnt<ND> *>(a.ptab);
    float2 *wbuf = reinterpret_cast<float2 *>(smem);                             // [2][S][NC][WP]
    const int nc = min(*a.n_cand, a.max_cand);
    const int n_chunks = (a.n_shifts + S - 1) / S;
    const int n_items = max(nc, 0) * n_chunks;
    int item = blockIdx.x;
    if (item >= n_items) return;
    PtItem<ND> cur = decode_item<ND, S>(a, item, n_chunks, lane);
    stage_item<ND, S, WP>(a, cur, wbuf, wid, lane);
    cp_async_commit();
    for (int k = 0; item < n_items; ++k, item += gridDim.x) {
        float2 *win = wbuf + (k & 1) * S * kShiftWords;
        // prefetch the next item into the other buffer (freed by the barrier that ended the
        // previous iteration), then wait for this item's copies
        const int nxt = item + gridDim.x;
        PtItem<ND> nit = cur;
        if (nxt < n_items) {
            nit = decode_item<ND, S>(a, nxt, n_chunks, lane);
            stage_item<ND, S, WP>(a, nit, wbuf + ((k + 1) & 1) * S * kShiftWords, wid, lane);
        }
        cp_async_commit();
        cp_async_wait<1>();
        __syncthreads();
        const int r = cur.r;
        // the reference sample (a nonzero mask implies a valid record)
        const float2 wr = cur.okmask ? a.snr[((int64_t)cur.t * ND + r) * a.pitch + cur.e] : make_float2(0.f, 0.f);
        const u64 wr2 = pack2(wr.x, wr.y);
        float best[S];
        int arg[S];
#pragma unroll
        for (int i = 0; i < S; ++i) {
            best[i] = -1.f;
            arg[i] = INT_MAX;
        }
        // the pixel loop for the first NA shifts of the chunk (NA a power of two): a short last
        // chunk (100 shifts in chunks of 16 end with 4) evaluates only the shifts it has
        auto scan = [&](auto na) {
            constexpr int NA = decltype(na)::value;
            const PtEnt<ND> *__restrict__ pr = ptab + (int64_t)r * a.n_pix;
            for (int p = tid; p < a.n_pix; p += kPtChunkThreads) {
                const PtEnt<ND> pe = pr[p];
                const u64 yb0 = mul2(pack2(pe.ur[0], pe.ur[0]), wr2), yb1 = mul2(pack2(pe.ur[1], pe.ur[1]), wr2);
                u64 U0[NC], U1[NC];
                const float *wq[NC];
#pragma unroll
                for (int q = 0; q < NC; ++q) {
                    U0[q] = pack2(pe.uq[q][0], pe.uq[q][0]);
                    U1[q] = pack2(pe.uq[q][1], pe.uq[q][1]);
                    wq[q] = reinterpret_cast<const float *>(win + q * WP + ((pe.idx >> (10 * q)) & 1023u));
                }
#pragma unroll
                for (int i = 0; i < NA; ++i) {
                    u64 y0 = yb0, y1 = yb1;
#pragma unroll
                    for (int q = 0; q < NC; ++q) {
                        const u64 w = lds64(wq[q] + 2 * i * kShiftWords);
                        y0 = fma2(U0[q], w, y0);
                        y1 = fma2(U1[q], w, y1);
                    }
                    const float2 m = unpack2(fma2(y1, y1, mul2(y0, y0)));
                    const float v = m.x + m.y;
                    if (v > best[i]) {
                        best[i] = v;
                        arg[i] = pe.p;
                    }
                }
            }
        };
        if (cur.okmask) {
            constexpr int S4 = S >= 4 ? S / 4 : 1, S2 = S >= 2 ? S / 2 : 1;
            if (cur.ns <= S4)
                scan(std::integral_constant<int, S4>{});
            else if (cur.ns <= S2)
                scan(std::integral_constant<int, S2>{});
            else
                scan(std::integral_constant<int, S>{});
        }
        // per shift, the warp's largest value (statistics are >= 0, so their bits order as
        // unsigned integers; no pixel counts as 0) and the lowest pixel holding it; lane i
        // keeps shift i's pair
        float rv = -1.f;
        int rp = INT_MAX;
#pragma unroll
        for (int i = 0; i < S; ++i) {
            const unsigned u = best[i] >= 0.f ? __float_as_uint(best[i]) : 0u;
            const unsigned m = __reduce_max_sync(0xffffffffu, u);
            const unsigned pm = __reduce_min_sync(0xffffffffu, u == m ? (unsigned)arg[i] : 0xFFFFFFFFu);
            rv = lane == i ? __uint_as_float(m) : rv;
            rp = lane == i ? (int)pm : rp;
        }
        if (lane < S) {
            s_v[wid][lane] = rv;
            s_p[wid][lane] = rp;
        }
        __syncthreads();
        if (tid < cur.ns) {
            const int i = tid;
            float bv = s_v[0][i];
            int bp = s_p[0][i];
#pragma unroll
            for (int w = 1; w < kWarps; ++w) take_pair(bv, bp, s_v[w][i], s_p[w][i]);
            const int64_t o = (int64_t)cur.c * a.n_shifts + cur.s_first + i;
            if (!((cur.okmask >> i) & 1u) || bp == INT_MAX) {
                a.max_stat[o] = __int_as_float(0x7fc00000);
                a.argmax[o] = -1;
                a.null_stat[o] = __int_as_float(0x7fc00000);
            } else {
                float nul = 0.f;
                if (ND > 2) {
                    const Entry en = tab[bp];
                    int offr = 0;
#pragma unroll
                    for (int J = 0; J < ND; ++J) offr = (J == r) ? en.off[J] : offr;
                    const float *un = a.u_null + (int64_t)bp * ND * (ND - 2);
                    for (int j = 0; j < ND - 2; ++j) {
                        float cr = 0.f, ci = 0.f;
#pragma unroll
                        for (int J = 0; J < ND; ++J) {
                            // companion slot of detector J and its window start (J != r)
                            const int q = (J < r) ? J : J - 1;
                            const int dm = (J < r) ? cur.dmn[J < NC ? J : 0] : cur.dmn[J > 0 ? J - 1 : 0];
                            const float2 w = (J == r) ? wr : win[i * kShiftWords + q * WP + en.off[J] - offr - dm];
                            const float u = un[J * (ND - 2) + j];
                            cr = fmaf(u, w.x, cr);
                            ci = fmaf(u, w.y, ci);
                        }
                        nul = fmaf(cr, cr, fmaf(ci, ci, nul));
                    }
                }
                a.max_stat[o] = bv;
                a.argmax[o] = bp;
                a.null_stat[o] = nul;
            }
        }
        __syncthreads();  // this buffer and the partial maxima are free again
        cur = nit;
    }
    cp_async_wait<0>();
}

// Resident blocks of a kernel for a dynamic shared-memory size (the opt-in limit is raised to
// max_smem once per kernel and device; both queries are cached per device).
template <typename K>
static int resident_blocks(K kern, int threads, size_t smem, int max_smem, int &n_sm, int &per_sm) {
    int dev = 0;
    SPIIR_CUDA_TRY(cudaGetDevice(&dev));
    SPIIR_TRY(set_max_dyn_smem((const void *)kern, max_smem));
    SPIIR_CUDA_TRY(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
    SPIIR_TRY(resident_blocks_per_sm((const void *)kern, threads, smem, &per_sm));
    return SPIIR_OK;
}

template <int ND, int S, int WP>
static int launch_chunked(const PointArgs &a, size_t smem, cudaStream_t stream) {
    auto kern = k_points_chunked<ND, S, WP>;
    int n_sm = 0, per_sm = 0;
    SPIIR_TRY(resident_blocks(kern, kPtChunkThreads, smem, kPtChunkSmem, n_sm, per_sm));
    const int64_t items = (int64_t)a.max_cand * ((a.n_shifts + S - 1) / S);
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(items, (int64_t)n_sm * std::max(per_sm, 1)));
    SPIIR_CUDA_TRY(launch_dependent(kern, dim3(grid), dim3(kPtChunkThreads), smem, stream, a));
    return SPIIR_OK;
}

// shifts per chunk: 1 for the zero-lag scan, else as many as keep the double-buffered windows
// within the shared memory of four blocks per SM (narrow windows) or two (wide ones)
static int chunk_shifts(int nd, int n_shifts) { return n_shifts == 1 ? 1 : (nd <= 3 ? 16 : 8); }

template <int ND, int WP>
static int dispatch_chunked_wp(const PointArgs &a, cudaStream_t stream) {
    const size_t win1 = sizeof(float2) * (ND - 1) * WP;  // one shift's windows
    switch (chunk_shifts(ND, a.n_shifts)) {
        case 1: return launch_chunked<ND, 1, WP>(a, 2 * win1, stream);
        case 8: return launch_chunked<ND, 8, WP>(a, 2 * 8 * win1, stream);
        default: return launch_chunked<ND, 16, WP>(a, 2 * 16 * win1, stream);
    }
}

template <int ND>
static int dispatch_chunked(const PointArgs &a, cudaStream_t stream) {
    return a.Wmax <= kPtWPNarrow ? dispatch_chunked_wp<ND, kPtWPNarrow>(a, stream)
                                 : dispatch_chunked_wp<ND, kPtWP>(a, stream);
}

template <int ND, bool SMEM_TAB>
static int launch_points(const PointArgs &a, size_t smem, cudaStream_t stream) {
    auto kern = k_points<ND, SMEM_TAB>;
    int n_sm = 0, per_sm = 0;
    SPIIR_TRY(resident_blocks(kern, kPtThreads, smem, kPtMaxSmem, n_sm, per_sm));
    const int64_t items = (int64_t)a.max_cand * a.n_shifts;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(items, (int64_t)n_sm * std::max(per_sm, 1)));
    SPIIR_CUDA_TRY(launch_dependent(kern, dim3(grid), dim3(kPtThreads), smem, stream, a));
    return SPIIR_OK;
}

template <int ND>
static int dispatch_points(const PointArgs &a, size_t smem, cudaStream_t stream) {
    return a.tab_bytes ? launch_points<ND, true>(a, smem, stream) : launch_points<ND, false>(a, smem, stream);
}

// The per-reference point entries of a sky (built once, after the relative delay ranges).
// Shared-memory wavefronts of one half-warp's 8-byte window reads, summed over the companions:
// for each companion, the largest number of distinct window entries that share a bank pair
// (entry mod 16; every window starts on a multiple of 16 entries).
static int half_warp_cost(const uint32_t *idx, int n, int NC) {
    int c = 0;
    for (int q = 0; q < NC; ++q) {
        int per_bank[16] = {0};
        for (int i = 0; i < n; ++i) {
            const uint32_t e = (idx[i] >> (10 * q)) & 1023u;
            bool seen = false;
            for (int j = 0; j < i && !seen; ++j) seen = ((idx[j] >> (10 * q)) & 1023u) == e;
            if (!seen) ++per_bank[e & 15];
        }
        c += *std::max_element(per_bank, per_bank + 16);
    }
    return c;
}

// Order of one chunk's pixels (key = packed window indices, value = pixel): sorted by key, then
// pixels exchanged between the half-warps' groups of 16 while that lowers the summed
// half_warp_cost (a fixed pseudo-random sequence of trial swaps, so the table is reproducible).
static void order_chunk(std::pair<uint64_t, int> *key, const uint32_t *idx_of_pixel, int n, int NC) {
    std::sort(key, key + n);
    const int G = (n + 15) / 16;
    if (G < 2) return;
    std::vector<uint32_t> idx(n);
    std::vector<int> cost(G);
    auto group_cost = [&](int g) { return half_warp_cost(&idx[16 * g], std::min(16, n - 16 * g), NC); };
    for (int i = 0; i < n; ++i) idx[i] = idx_of_pixel[key[i].second];
    for (int g = 0; g < G; ++g) cost[g] = group_cost(g);
    uint64_t x = 0x9E3779B97F4A7C15ull;
    for (int trial = 0; trial < 40 * n; ++trial) {
        x = x * 6364136223846793005ull + 1442695040888963407ull;
        const int i = (int)((x >> 33) % (uint64_t)n), j = (int)((x >> 13) % (uint64_t)n);
        const int gi = i / 16, gj = j / 16;
        if (gi == gj) continue;
        std::swap(idx[i], idx[j]);
        const int ci = group_cost(gi), cj = group_cost(gj);
        if (ci + cj <= cost[gi] + cost[gj]) {
            std::swap(key[i], key[j]);
            cost[gi] = ci;
            cost[gj] = cj;
        } else {
            std::swap(idx[i], idx[j]);
        }
    }
}

template <int ND>
static int build_point_table(spiir_sky_s *sky) {
    const int P = sky->n_pix;
    std::vector<PtEnt<ND>> h((size_t)ND * P);
    for (int r = 0; r < ND; ++r) {
        std::vector<std::pair<uint64_t, int>> key(P);
        std::vector<uint32_t> idx(P);
        for (int p = 0; p < P; ++p) {
            const int32_t *dl = &sky->h_delays[(size_t)p * ND];
            uint64_t k = 0;
            idx[p] = 0;
            for (int q = 0; q < ND - 1; ++q) {
                const int J = q < r ? q : q + 1;
                const uint32_t e = (uint32_t)(dl[J] - dl[r] - sky->rel_min[r * ND + J]);
                k = (k << 10) | (uint64_t)e;
                idx[p] |= e << (10 * q);
            }
            key[p] = {k, p};
        }
        for (int c0 = 0; c0 < P; c0 += kPtChunkThreads)
            order_chunk(&key[c0], idx.data(), std::min(P - c0, kPtChunkThreads), ND - 1);
        for (int i = 0; i < P; ++i) {
            const int p = key[i].second;
            PtEnt<ND> &e = h[(size_t)r * P + i];
            const int32_t *dl = &sky->h_delays[(size_t)p * ND];
            const float *us = &sky->h_usig[(size_t)p * ND * 2];
            e.ur[0] = us[2 * r];
            e.ur[1] = us[2 * r + 1];
            e.idx = 0;
            for (int q = 0; q < ND - 1; ++q) {
                const int J = q < r ? q : q + 1;
                e.uq[q][0] = us[2 * J];
                e.uq[q][1] = us[2 * J + 1];
                e.idx |= (uint32_t)(dl[J] - dl[r] - sky->rel_min[r * ND + J]) << (10 * q);
            }
            e.p = p;
        }
    }
    void *d = nullptr;
    SPIIR_TRY(dev_alloc(&d, h.size() * sizeof(PtEnt<ND>), "candidate point table"));
    if (cudaMemcpy(d, h.data(), h.size() * sizeof(PtEnt<ND>), cudaMemcpyHostToDevice) != cudaSuccess) {
        dev_free(d);
        return fail(SPIIR_ECUDA, "copy of the candidate point table failed");
    }
    sky->pt_tab = d;
    return SPIIR_OK;
}

}  // namespace spiir

using namespace spiir;

static int64_t n_seconds(int64_t n, int per_second) { return (n + per_second - 1) / per_second; }

extern "C" int spiir_select_workspace_bytes(int T, int n_det, int64_t n, int per_second, size_t *bytes) {
    clear_error();
    if (!bytes) return fail(SPIIR_EINVAL, "bytes is NULL");
    if (T < 1 || n_det < 1 || n < 1 || per_second < 1)
        return fail(SPIIR_EINVAL, "n_templates = %d, n_det = %d, n = %lld, per_second = %d", T, n_det, (long long)n,
                    per_second);
    // slots, per-sample keys and the compaction's block counter
    *bytes = sizeof(u64) * ((size_t)n_det * ((size_t)T * (size_t)n_seconds(n, per_second) + (size_t)n) + 1);
    return SPIIR_OK;
}

extern "C" int spiir_select_candidates(int T, int n_det, const float *snr, int64_t pitch, int64_t off, int64_t n,
                                       float threshold, int per_second, void *workspace, size_t workspace_bytes,
                                       int32_t *cand, int max_cand, int32_t *n_cand, void *stream) {
    clear_error();
    if (T < 1 || n_det < 1 || n < 1 || per_second < 1)
        return fail(SPIIR_EINVAL, "n_templates = %d, n_det = %d, n = %lld, per_second = %d", T, n_det, (long long)n,
                    per_second);
    if (n_det > 65535) return fail(SPIIR_EINVAL, "n_det = %d above 65535", n_det);
    if (n > INT_MAX) return fail(SPIIR_EINVAL, "n = %lld above 2^31 - 1", (long long)n);
    if (off < 0 || pitch < off + n)
        return fail(SPIIR_EINVAL, "entries [%lld, %lld) outside the row pitch %lld", (long long)off,
                    (long long)(off + n), (long long)pitch);
    if (max_cand < 0) return fail(SPIIR_EINVAL, "max_cand = %d", max_cand);
    if (!snr || !workspace || !n_cand || (max_cand > 0 && !cand)) return fail(SPIIR_EINVAL, "NULL pointer");
    if (((uintptr_t)snr) % 8 || ((uintptr_t)workspace) % 8 || (cand && ((uintptr_t)cand) % 16))
        return fail(SPIIR_EINVAL, "snr and workspace must be 8-byte aligned, cand 16-byte aligned");
    if (!(threshold >= 0.f) || !std::isfinite(threshold)) return fail(SPIIR_EINVAL, "threshold must be finite and >= 0");
    const int64_t n_sec = n_seconds(n, per_second);
    const int64_t n_cols = (n + 31) / 32, n_chunks = (T + kSelTaskT - 1) / kSelTaskT;
    if ((int64_t)n_det * n > INT_MAX || (int64_t)n_det * T * n_sec > INT_MAX || n_cols * n_det * n_chunks > INT_MAX)
        return fail(SPIIR_EINVAL, "n_det x n and n_det x n_templates x seconds must be below 2^31");
    size_t need = 0;
    SPIIR_TRY(spiir_select_workspace_bytes(T, n_det, n, per_second, &need));
    if (workspace_bytes < need)
        return fail(SPIIR_EINVAL, "workspace of %zu bytes, %zu needed", workspace_bytes, need);
    const float thr2 = threshold * threshold;  // FP32, round to nearest (as the per-sample |z|^2)
    cudaStream_t st = (cudaStream_t)stream;
    u64 *slots = static_cast<u64 *>(workspace);
    u64 *keys = slots + (size_t)n_det * T * n_sec;
    unsigned *done = reinterpret_cast<unsigned *>(keys + (size_t)n_det * n);
    const int64_t n_tasks = n_cols * n_det * n_chunks;
    const int blocks = (int)((n_tasks + kSelBlock / 32 - 1) / (kSelBlock / 32));
    k_select<<<blocks, kSelBlock, 0, st>>>(reinterpret_cast<const float2 *>(snr), pitch, off, T, n_det, (int)n,
                                           (int)n_cols, (int)n_chunks, keys);
    SPIIR_CUDA_TRY(cudaGetLastError());
    // programmatic dependent launch: the compaction blocks are scheduled while the selection
    // drains and wait for its completion
    SPIIR_CUDA_TRY(launch_dependent(k_compact, dim3((unsigned)(((int64_t)n_det * n + kCompThreads - 1) / kCompThreads)),
                                    dim3(kCompThreads), 0, st, keys, (int)n, n_det, T, thr2, per_second, slots,
                                    (int)n_sec, done, reinterpret_cast<int4 *>(cand), max_cand, n_cand));
    return SPIIR_OK;
}

extern "C" int spiir_coherent_candidates(spiir_sky_t sky, int T, const float *snr, int64_t pitch, int64_t off,
                                         const int32_t *cand, const int32_t *n_cand, int max_cand, int first_shift,
                                         int n_shifts, int shift_step, float *max_stat, int32_t *argmax,
                                         float *null_stat, void *stream) {
    clear_error();
    if (!sky) return fail(SPIIR_EINVAL, "sky is NULL");
    if (T < 1 || max_cand < 0 || n_shifts < 1 || first_shift < 0 || shift_step < 0 || off < 0 || pitch < 1)
        return fail(SPIIR_EINVAL,
                    "n_templates = %d, max_cand = %d, first_shift = %d, n_shifts = %d, shift_step = %d, "
                    "offset = %lld, pitch = %lld",
                    T, max_cand, first_shift, n_shifts, shift_step, (long long)off, (long long)pitch);
    if ((int64_t)max_cand * n_shifts > INT_MAX) return fail(SPIIR_EINVAL, "max_cand x n_shifts above 2^31 - 1");
    if (!snr || !n_cand || (max_cand > 0 && (!cand || !max_stat || !argmax || !null_stat)))
        return fail(SPIIR_EINVAL, "NULL pointer");
    if (((uintptr_t)snr) % 8 || (cand && ((uintptr_t)cand) % 16))
        return fail(SPIIR_EINVAL, "snr must be 8-byte aligned, cand 16-byte aligned");
    if (max_cand == 0) return SPIIR_OK;
    const int ND = sky->n_det;
    PointArgs a{};
    a.snr = reinterpret_cast<const float2 *>(snr);
    a.pitch = pitch;
    a.off = off;
    a.n_templates = T;
    a.cand = reinterpret_cast<const int4 *>(cand);
    a.n_cand = n_cand;
    a.max_cand = max_cand;
    a.first_shift = first_shift;
    a.n_shifts = n_shifts;
    a.step = shift_step;
    a.table = sky->table;
    a.u_null = sky->u_null;
    a.n_pix = sky->n_pix;
    a.H = sky->halo;
    if (sky->rel_min.empty()) {
        std::vector<int> mn(ND * ND), mx(ND * ND);
        for (int r = 0; r < ND; ++r)
            for (int J = 0; J < ND; ++J) {
                int lo = INT_MAX, hi = INT_MIN;
                for (int p = 0; p < sky->n_pix; ++p) {
                    const int d = sky->h_delays[(size_t)p * ND + J] - sky->h_delays[(size_t)p * ND + r];
                    lo = std::min(lo, d);
                    hi = std::max(hi, d);
                }
                mn[r * ND + J] = lo;
                mx[r * ND + J] = hi;
            }
        sky->rel_min = mn;
        sky->rel_max = mx;
    }
    int Wmax = 1;
    for (int r = 0; r < ND; ++r)
        for (int J = 0; J < ND; ++J) {
            a.dmin[r][J] = sky->rel_min[r * ND + J];
            a.dmax[r][J] = sky->rel_max[r * ND + J];
            Wmax = std::max(Wmax, a.dmax[r][J] - a.dmin[r][J] + 1);
        }
    if (!sky->pt_tab) {
        switch (ND) {
            case 2: SPIIR_TRY(build_point_table<2>(sky)); break;
            case 3: SPIIR_TRY(build_point_table<3>(sky)); break;
            case 4: SPIIR_TRY(build_point_table<4>(sky)); break;
            default: break;
        }
    }
    a.ptab = sky->pt_tab;
    a.Wmax = Wmax;
    a.max_stat = max_stat;
    a.argmax = argmax;
    a.null_stat = null_stat;
    cudaStream_t st = (cudaStream_t)stream;
    {
        const int S = chunk_shifts(ND, n_shifts);
        const size_t chunk_bytes = 2 * sizeof(float2) * (size_t)S * (ND - 1) * kPtWP;  // double-buffered windows
        const int64_t items = (int64_t)max_cand * ((n_shifts + S - 1) / S);              // 32-bit item numbers
        if (Wmax <= kPtWP && chunk_bytes <= (size_t)kPtChunkSmem && items < (1 << 30)) {
            a.tab_bytes = 0;
            switch (ND) {
                case 2: return dispatch_chunked<2>(a, st);
                case 3: return dispatch_chunked<3>(a, st);
                case 4: return dispatch_chunked<4>(a, st);
                default: return fail(SPIIR_EUNSUPPORTED, "n_det = %d", ND);
            }
        }
    }
    const size_t win_bytes = sizeof(float2) * (size_t)ND * Wmax;
    a.tab_bytes = (sky->table_bytes + win_bytes <= (size_t)kPtMaxSmem) ? sky->table_bytes : 0;
    const size_t smem = a.tab_bytes + win_bytes;
    if (smem > (size_t)kPtMaxSmem) return fail(SPIIR_EUNSUPPORTED, "SNR windows of %zu bytes", win_bytes);
    switch (ND) {
        case 2: return dispatch_points<2>(a, smem, st);
        case 3: return dispatch_points<3>(a, smem, st);
        case 4: return dispatch_points<4>(a, smem, st);
        default: return fail(SPIIR_EUNSUPPORTED, "n_det = %d", ND);
    }
}
