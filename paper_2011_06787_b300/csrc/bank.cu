// SPIIR filter bank (Sec. II.B.1, Eq. (zk), per-filter reading):
//     y_l[k] = a1_l y_l[k-1] + b0_l x_I[k - d_l],     z_{t,I}[k] = sum_{l in t} y_l[k].
//
// Device mapping (K1):
//   * A thread ("lane") owns S filters of one template and keeps their coefficients and
//     complex states in registers as packed FP32 pairs (two filters per f32x2 register),
//     so one packed update costs 8 FP32-pipe operations for two filter-samples.
//   * Templates occupy contiguous lane ranges; whole templates are packed into thread
//     blocks of NL lanes (best-fit decreasing), so no template straddles two blocks.
//   * blockIdx.y selects the detector.  The strain window of a time tile plus the maximum
//     delay is copied into shared memory by one bulk asynchronous copy completed on an
//     mbarrier.
//   * Every lane writes its per-step partial sum (over its S filters) to a shared buffer
//     of R steps.  After R steps each warp sums its 32 rows column by column, split at
//     template boundaries (warp-uniform), and one more pass adds the pieces of templates
//     that span several warps and writes z with coalesced stores.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <climits>
#include <map>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "bank.cuh"

namespace spiir {

// ---------------------------------------------------------------------------------------
// Kernel

// Shared-memory layout of one block: the mbarrier at offset 0, the strain window at
// kBankSmemHead, the reduction buffer at a.red_offset.

// Pairwise sum of N packed pairs (N a power of two).
template <int N>
__device__ __forceinline__ u64 tree_sum2(const u64 (&v)[N]) {
    u64 w[N];
#pragma unroll
    for (int i = 0; i < N; ++i) w[i] = v[i];
#pragma unroll
    for (int h = N / 2; h >= 1; h /= 2) {
#pragma unroll
        for (int i = 0; i < h; ++i) w[i] = add2(w[i], w[i + h]);
    }
    return w[0];
}

// Row stride (float2 entries) of the per-step sums in the reduction buffer: R + 2, even, so
// that the sums of steps 2i and 2i + 1 of a row form one aligned 16-byte store.
__host__ __device__ constexpr int bank_red_stride(int R) { return R + 2; }

// One block's work: template block `cta` of bank `a` for detector `det` over the whole call.
// Returns false when a bounded wait ran out (every thread of the block returns false).
template <int S, int NL, int R>
__device__ __forceinline__ bool bank_block(const BankArgs &a, const int cta, const int det, unsigned char *smem,
                                           uint64_t *bar, uint32_t &phase) {
    constexpr int NP = S / 2;
    constexpr int NW = NL / 32;
    float *xw = reinterpret_cast<float *>(smem + kBankSmemHead);
    float2 *red = reinterpret_cast<float2 *>(smem + a.red_offset);

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
#ifdef SPIIR_CHECKED
    {
        int bad = 0;
        if (cta < 0 || cta >= a.n_cta_total) bad = 1;
        else if (((int64_t)cta * (S / 2) + S / 2) * NL > a.n_pairs_total) bad = 2;
        else if (a.seg_off && (a.seg_off[cta] < 0 || a.seg_off[cta + 1] > a.n_segs_total)) bad = 3;
        if (__syncthreads_or(bad)) {
            if (bad) report_bounds(a.status, bad);
            return false;
        }
    }
#endif
    const int active = a.cta_active[cta];
    const bool busy = (warp * 32) < active;

    // coefficients and states -> registers
    u64 are[NP], aim[NP], naim[NP], bre[NP], bim[NP], yre[NP], yim[NP];
    int dof[S];
    const int64_t pbase = (int64_t)cta * NP * NL + tid;
    float4 *st = a.state + (int64_t)det * a.state_det_stride + pbase;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        float2 v;
        v = a.are[pbase + (int64_t)p * NL];
        are[p] = pack2(v.x, v.y);
        v = a.aim[pbase + (int64_t)p * NL];
        aim[p] = pack2(v.x, v.y);
        naim[p] = neg2(aim[p]);
        v = a.bre[pbase + (int64_t)p * NL];
        bre[p] = pack2(v.x, v.y);
        v = a.bim[pbase + (int64_t)p * NL];
        bim[p] = pack2(v.x, v.y);
        float4 y = st[(int64_t)p * NL];
        yre[p] = pack2(y.x, y.y);
        yim[p] = pack2(y.z, y.w);
    }
    // the block's strain window: x[k0 - dhi, k0 - dhi + span + nt) of each tile (dhi, span
    // multiples of 4), which holds every delayed sample its filters read
    const int2 win = a.cta_win[cta];
#pragma unroll
    for (int s = 0; s < S; ++s) dof[s] = win.x - a.delay[((int64_t)cta * S + s) * NL + tid];

    // segment tables of this block
    const int seg0 = a.seg_off[cta];
    const int nseg = a.seg_off[cta + 1] - seg0;
    const int wfirst = a.wfirst[cta * NW + warp];
    const float *xsrc = a.xbuf + (int64_t)det * a.xpitch + (a.D_pad - win.x);

    for (int64_t k0 = 0; k0 < a.n; k0 += a.c_tile) {
        const int nt = (int)min((int64_t)a.c_tile, a.n - k0);
        const uint32_t bytes = (uint32_t)(win.y + ((nt + 3) & ~3)) * 4u;
#ifdef SPIIR_CHECKED
        {
            int bad = 0;
            if (win.x > a.D_pad || win.y > win.x || win.y < 0) bad = 9;
            if ((int64_t)det * a.xpitch + (a.D_pad - win.x) + k0 + bytes / 4 > a.x_elems) bad = 4;
            if (kBankSmemHead + bytes > a.red_offset) bad = 5;
            for (int s = 0; s < S; ++s)
                if (dof[s] < 0 || dof[s] > win.y) bad = 6;
            if (__syncthreads_or(bad)) {
                if (bad) report_bounds(a.status, bad);
                return false;
            }
        }
#endif
        __syncthreads();  // all reads of the previous window are done
        if (tid == 0) bulk_load(xw, xsrc + k0, bytes, bar);
        const bool ok = mbar_wait(bar, phase);
        if (__syncthreads_or(!ok)) {
            // bounded wait ran out: record it, give the copy one more bounded wait, leave
            if (tid == 0) {
                report_timeout(a.status);
                mbar_wait(bar, phase);
            }
            return false;
        }
        phase ^= 1u;

        for (int kb = 0; kb < nt; kb += R) {
            const int nr = min(R, nt - kb);
            if (busy) {
                const float *xp[S];
#pragma unroll
                for (int s = 0; s < S; ++s) xp[s] = xw + dof[s] + kb;
                constexpr int RS = bank_red_stride(R);
                float2 *rrow = red + tid * RS;
                auto step = [&](int r) -> float2 {
#pragma unroll
                    for (int p = 0; p < NP; ++p) {
                        const u64 X = pack2(xp[2 * p][r], xp[2 * p + 1][r]);
                        u64 t = fma2(are[p], yre[p], mul2(bre[p], X));  // a.re y.re + b.re x
                        u64 u = fma2(are[p], yim[p], mul2(bim[p], X));  // a.re y.im + b.im x
                        const u64 nr_ = fma2(naim[p], yim[p], t);       // - a.im y.im
                        const u64 ni_ = fma2(aim[p], yre[p], u);        // + a.im y.re
                        yre[p] = nr_;
                        yim[p] = ni_;
                    }
                    // the lane's sum over its S filters as a pairwise tree (shorter dependency
                    // chains than a running sum)
                    const float2 ar = unpack2(tree_sum2<NP>(yre)), ai = unpack2(tree_sum2<NP>(yim));
                    return make_float2(ar.x + ar.y, ai.x + ai.y);
                };
                if (nr == R) {
#pragma unroll
                    for (int r = 0; r < R; r += 2) {
                        const float2 s0 = step(r), s1 = step(r + 1);
                        *reinterpret_cast<float4 *>(rrow + r) = make_float4(s0.x, s0.y, s1.x, s1.y);
                    }
                } else {
#pragma unroll 1
                    for (int r = 0; r < nr; ++r) rrow[r] = step(r);
                }
            }
            __syncwarp();
            // pass 1: each warp sums its own rows per column, split at template boundaries;
            // piece j of the warp overwrites row 32*warp + j (a row it has already read).
            // Only rows written by the same warp are read, so a warp barrier suffices.
            // With R < 32 some lanes have no column; with R = 64 each lane has two.
            // Lane c owns columns c, c + 32, ... below R.
            // The (re, im) partial sums are added as packed pairs, rows in order (the same
            // rounding as two scalar additions).
            u64 *red2 = reinterpret_cast<u64 *>(red);
            for (int col = lane; busy && wfirst >= 0 && col < R; col += 32) {
                constexpr int RS = bank_red_stride(R);
                u64 *colp = red2 + (warp * 32) * RS + col;
                int j = 0;
                for (int sg = wfirst; sg < nseg; ++sg) {
                    const int4 g = a.segs[seg0 + sg];
                    const int lo = max(g.y, warp * 32) - warp * 32;
                    const int hi = min(g.z, warp * 32 + 32) - warp * 32;
                    if (hi <= lo) break;
#ifdef SPIIR_CHECKED
                    if ((warp * 32 + hi - 1) * RS + col >= NL * RS) {
                        report_bounds(a.status, 8);
                        break;
                    }
#endif
                    u64 acc = 0;  // (+0, +0)
                    const u64 *rp = colp + lo * RS;
#pragma unroll 8
                    for (int i = lo; i < hi; ++i, rp += RS) acc = add2(acc, *rp);
                    colp[j * RS] = acc;
                    ++j;
                }
            }
            __syncthreads();
            // pass 2: add the pieces of each template over the warps it spans, write z
            for (int o = tid; o < nseg * R; o += NL) {
                const int sg = o / R, r = o % R;
                if (r >= nr) continue;
                const int4 g = a.segs[seg0 + sg];
                u64 acc = 0;
                for (int w = g.y >> 5; w <= (g.z - 1) >> 5; ++w)
                    acc = add2(acc, red2[(w * 32 + (sg - a.wfirst[cta * NW + w])) * bank_red_stride(R) + r]);
                // a template's first delay piece writes z; its later pieces write zpart rows
                float2 *zrow = g.w ? a.zpart + ((int64_t)g.x * a.n_det + det) * a.zpart_pitch
                                   : a.z + ((int64_t)g.x * a.n_det + det) * a.zpitch;
#ifdef SPIIR_CHECKED
                if (g.w ? ((int64_t)g.x * a.n_det + det) * a.zpart_pitch + k0 + kb + r >= a.zpart_elems
                        : ((int64_t)g.x * a.n_det + det) * a.zpitch + k0 + kb + r >= a.z_elems) {
                    report_bounds(a.status, 7);
                    continue;
                }
#endif
                zrow[k0 + kb + r] = unpack2(acc);
            }
            __syncthreads();
        }
    }
    // states back to global memory
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        const float2 r = unpack2(yre[p]), i = unpack2(yim[p]);
        st[(int64_t)p * NL] = make_float4(r.x, r.y, i.x, i.y);
    }
    return true;
}

// The default shape (8 filters per lane, 128 lanes) asks for 5 resident blocks: the compiler
// then keeps it at 92 registers without spills (117 otherwise).
template <int S, int NL, int R>
__global__ void __launch_bounds__(NL, (S == 8 && NL == 128) ? 5 : 1) k_filter_bank(const __grid_constant__ BankArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
    if (threadIdx.x == 0) mbar_init(bar, 1);
    __syncthreads();
    uint32_t phase = 0;
    bank_block<S, NL, R>(a, blockIdx.x, blockIdx.y, smem, bar, phase);
}

// Persistent form: a grid of resident blocks takes (bank, block, detector) work items from a
// shared counter (atomic fetch-and-add, no waiting) in the order of the item list, so that
// banks of uneven size and different rates share one launch.  The default shape asks for four
// resident blocks (at most 128 registers), which the multirate banks' shared memory allows.
template <int S, int NL, int R>
__global__ void __launch_bounds__(NL, (S == 8 && NL == 128) ? 4 : 1)
    k_filter_bank_persistent(const __grid_constant__ PersistArgs p) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int item_s;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
    if (threadIdx.x == 0) mbar_init(bar, 1);
    __syncthreads();
    uint32_t phase = 0;
    for (;;) {
        if (threadIdx.x == 0) item_s = atomicAdd(p.counter, 1);
        __syncthreads();
        const int item = item_s;
        __syncthreads();
        if (item >= p.n_items) break;
        const int4 it = p.items[item];
        if (!bank_block<S, NL, R>(p.banks[it.x], it.y, it.z, smem, bar, phase)) break;
    }
}

template <int S, int NL, int R>
static int launch_bank(const BankArgs &a, int n_cta, int n_det, size_t smem, cudaStream_t stream) {
    SPIIR_TRY(set_max_dyn_smem((const void *)k_filter_bank<S, NL, R>, kBankMaxSmem));
    k_filter_bank<S, NL, R><<<dim3(n_cta, n_det), NL, smem, stream>>>(a);
    SPIIR_CUDA_TRY(cudaGetLastError());
    return SPIIR_OK;
}

template <int S, int NL>
static int launch_bank_r(const BankArgs &a, int R, int n_cta, int n_det, size_t smem, cudaStream_t s) {
    switch (R) {
        case 16: return launch_bank<S, NL, 16>(a, n_cta, n_det, smem, s);
        case 20: return launch_bank<S, NL, 20>(a, n_cta, n_det, smem, s);
        case 64: return launch_bank<S, NL, 64>(a, n_cta, n_det, smem, s);
        default: return launch_bank<S, NL, 32>(a, n_cta, n_det, smem, s);
    }
}

template <int S>
static int launch_bank_nl(const BankArgs &a, int NL, int R, int n_cta, int n_det, size_t smem, cudaStream_t s) {
    return NL == 128 ? launch_bank_r<S, 128>(a, R, n_cta, n_det, smem, s) : launch_bank_r<S, 256>(a, R, n_cta, n_det, smem, s);
}

static int launch_bank_any(const spiir_bank_s *b, const BankArgs &a, size_t smem, cudaStream_t s) {
    switch (b->S) {
        case 4: return launch_bank_nl<4>(a, b->NL, b->R, b->n_cta, b->n_det, smem, s);
        case 8: return launch_bank_nl<8>(a, b->NL, b->R, b->n_cta, b->n_det, smem, s);
        default: return launch_bank_nl<16>(a, b->NL, b->R, b->n_cta, b->n_det, smem, s);
    }
}

size_t bank_red_offset(const spiir_bank_s *b) {
    return kBankSmemHead + (size_t)(((b->win_max + b->c_tile + 3) / 4) * 4 * sizeof(float) + 127) / 128 * 128;
}

size_t bank_smem_bytes(const spiir_bank_s *b) {
    return bank_red_offset(b) + (size_t)b->NL * bank_red_stride(b->R) * sizeof(float2);
}

// ---------------------------------------------------------------------------------------
// Host: packing

// A delay piece: the filters of one template whose delays fall in one delay bin.  A bank
// without bins has one piece per template.  The first piece of a template writes the
// template's z row; its later pieces write rows of zpart, added into z after the launch.
struct Piece {
    int t = 0;                   // template
    int row = 0;                 // z row (w = 0) or zpart row (w = 1)
    int w = 0;
    std::vector<int64_t> filt;   // filter indices, ascending
    int lanes = 1;
};

// Place the filters of the pieces of block c into (lane, slot) cells.  In the kernel, the
// 32 lanes of a warp load x[k - d] for the same slot in one shared-memory instruction; two
// different delays with the same residue mod 32 hit the same bank and serialise.  Rows
// (warp, slot) are therefore filled greedily with distinct residues: each cell takes a filter
// of its own piece from the residue class with the most filters left that is still free in
// the row, most loaded pieces first.  When every remaining residue of a piece is taken
// in the row, the cell stays empty (zero coefficients) if the piece has spare cells, and
// otherwise accepts a conflict.  Empty cells reuse a delay already read in the row (dfill,
// a delay of the block, when the row has none), so they cost no extra bank access and stay
// inside the block's window.
static void assign_cells(spiir_bank_s *b, int c, const std::vector<int> &lane_p, const std::vector<Piece> &pcs,
                         const std::vector<int> &members, int32_t dfill) {
    const int S = b->S, NL = b->NL, NP = S / 2;
    std::map<int, std::vector<std::vector<int64_t>>> pools;  // piece -> residue -> filters
    std::map<int, int64_t> rem_f, rem_c;
    for (int q : members) {
        auto &P = pools[q];
        P.assign(32, {});
        for (int64_t l : pcs[q].filt) P[b->delay[l] & 31].push_back(l);
        // pop from the back: keep a deterministic order within a residue class
        for (auto &v : P) std::reverse(v.begin(), v.end());
        rem_f[q] = (int64_t)pcs[q].filt.size();
        int64_t ln = 0;
        for (int j = 0; j < NL; ++j) ln += (lane_p[j] == q);
        rem_c[q] = ln * S;
    }
    auto place = [&](int ln, int s, int64_t l, int32_t d) {
        const int64_t slot = ((int64_t)c * S + s) * NL + ln;
        b->h_delay[slot] = d;
        if (l < 0) return;
        b->slot_of_filter[l] = slot;
        const size_t pi = ((size_t)c * NP + s / 2) * NL + ln;
        float2 *ar = &b->h_are[pi], *ai = &b->h_aim[pi], *br = &b->h_bre[pi], *bi = &b->h_bim[pi];
        if (s % 2 == 0) {
            ar->x = b->a1[2 * l]; ai->x = b->a1[2 * l + 1];
            br->x = b->b0[2 * l]; bi->x = b->b0[2 * l + 1];
        } else {
            ar->y = b->a1[2 * l]; ai->y = b->a1[2 * l + 1];
            br->y = b->b0[2 * l]; bi->y = b->b0[2 * l + 1];
        }
    };
    for (int s = 0; s < S; ++s) {
        for (int w = 0; w < NL / 32; ++w) {
            std::vector<int> ls;
            for (int j = 32 * w; j < 32 * w + 32; ++j)
                if (lane_p[j] >= 0) ls.push_back(j);
            if (ls.empty()) continue;
            std::stable_sort(ls.begin(), ls.end(), [&](int x, int y) {
                const int qx = lane_p[x], qy = lane_p[y];
                return (double)rem_f[qx] / std::max<int64_t>(1, rem_c[qx]) >
                       (double)rem_f[qy] / std::max<int64_t>(1, rem_c[qy]);
            });
            uint32_t used = 0;
            int32_t row_delay = -1;
            std::vector<int> empty;
            for (int ln : ls) {
                const int q = lane_p[ln];
                auto &P = pools[q];
                rem_c[q] -= 1;
                if (rem_f[q] == 0) {
                    empty.push_back(ln);
                    continue;
                }
                int best = -1;
                for (int r = 0; r < 32; ++r)
                    if (!P[r].empty() && !(used >> r & 1u) && (best < 0 || P[r].size() > P[best].size())) best = r;
                if (best < 0) {
                    if (rem_f[q] <= rem_c[q]) {
                        empty.push_back(ln);
                        continue;
                    }
                    for (int r = 0; r < 32; ++r)
                        if (!P[r].empty() && (best < 0 || P[r].size() > P[best].size())) best = r;
                }
                const int64_t l = P[best].back();
                P[best].pop_back();
                rem_f[q] -= 1;
                used |= 1u << best;
                if (row_delay < 0) row_delay = b->delay[l];
                place(ln, s, l, b->delay[l]);
            }
            for (int ln : empty) place(ln, s, -1, row_delay < 0 ? dfill : row_delay);
            // unused lanes of a busy warp run zero filters too: read the same address
            for (int j = 32 * w; j < 32 * w + 32; ++j)
                if (lane_p[j] < 0) place(j, s, -1, row_delay < 0 ? dfill : row_delay);
        }
    }
}

// Cut the templates into delay pieces (one per template without bins) and pack the pieces of
// each bin into blocks, best-fit decreasing: no piece straddles two blocks, and a block holds
// one bin only, so its window spans at most the bin width plus the tile.
int bank_pack(spiir_bank_s *b) {
    const int T = b->T;
    const int S = b->S;
    const int NL = b->NL;
    const int NW = NL / 32;
    for (int t = 0; t < T; ++t) {
        const int64_t f = b->offsets[t + 1] - b->offsets[t];
        if ((f + S - 1) / S > NL)
            return fail(SPIIR_EUNSUPPORTED, "template %d has %lld filters; at most %d per template", t,
                        (long long)f, NL * S);
    }
    std::vector<Piece> pcs;
    std::map<int, std::vector<int>> by_bin;   // bin -> pieces
    b->h_red_t.clear();
    b->h_red_off.assign(1, 0);
    int n_part = 0;
    for (int t = 0; t < T; ++t) {
        std::map<int, std::vector<int64_t>> bins;
        for (int64_t l = b->offsets[t]; l < b->offsets[t + 1]; ++l)
            bins[b->dbin > 0 ? b->delay[l] / b->dbin : 0].push_back(l);
        if (bins.empty()) bins[0];  // a template without filters still writes its (zero) row
        bool first = true;
        for (auto &kv : bins) {
            Piece p;
            p.t = t;
            p.filt = std::move(kv.second);
            p.lanes = (int)std::max<int64_t>(1, ((int64_t)p.filt.size() + S - 1) / S);
            if (first) {
                p.row = t;
                p.w = 0;
            } else {
                p.row = n_part++;
                p.w = 1;
            }
            by_bin[kv.first].push_back((int)pcs.size());
            pcs.push_back(std::move(p));
            first = false;
        }
        if (bins.size() > 1) {
            b->h_red_t.push_back(t);
            b->h_red_off.push_back(n_part);
        }
    }
    b->n_part = n_part;
    // best-fit decreasing within each bin: the largest pieces first into the fullest block that
    // still has room
    std::vector<std::vector<int>> members;
    for (auto &kv : by_bin) {
        std::vector<int> order = kv.second;
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return pcs[x].lanes > pcs[y].lanes; });
        std::multimap<int, int> by_free;  // free lanes -> block
        std::vector<int> used;
        const size_t c_first = members.size();
        for (int q : order) {
            auto it = by_free.lower_bound(pcs[q].lanes);
            int c;
            if (it == by_free.end()) {
                c = (int)members.size();
                members.emplace_back();
                used.push_back(0);
            } else {
                c = it->second;
                by_free.erase(it);
            }
            members[c].push_back(q);
            used[c - c_first] += pcs[q].lanes;
            by_free.emplace(NL - used[c - c_first], c);
        }
    }
    const int n_cta = (int)members.size();
    b->n_cta = n_cta;
    const int NP = S / 2;
    const int64_t n_slots = (int64_t)n_cta * S * NL;
    b->h_are.assign((size_t)n_cta * NP * NL, make_float2(0, 0));
    b->h_aim = b->h_are;
    b->h_bre = b->h_are;
    b->h_bim = b->h_are;
    b->h_delay.assign((size_t)n_slots, 0);
    b->slot_of_filter.assign((size_t)b->F, -1);
    b->h_segs.clear();
    b->h_seg_off.assign(n_cta + 1, 0);
    b->h_wfirst.assign((size_t)n_cta * NW, -1);
    b->h_active.assign(n_cta, 0);
    b->h_win.assign(n_cta, make_int2(0, 0));
    b->win_max = 0;
    std::vector<int> lane_p(NL);
    for (int c = 0; c < n_cta; ++c) {
        // within a block, pieces in ascending template order
        std::sort(members[c].begin(), members[c].end(), [&](int x, int y) { return pcs[x].t < pcs[y].t; });
        // the block's window: its delays rounded out to multiples of 4 (16-byte copies)
        int32_t dmin = INT32_MAX, dmax = -1;
        for (int q : members[c])
            for (int64_t l : pcs[q].filt) {
                dmin = std::min(dmin, b->delay[l]);
                dmax = std::max(dmax, b->delay[l]);
            }
        if (dmax < 0) dmin = dmax = 0;
        const int dhi = (dmax + 3) / 4 * 4, dlo = dmin / 4 * 4;
        b->h_win[c] = make_int2(dhi, dhi - dlo);
        b->win_max = std::max(b->win_max, dhi - dlo);
        std::fill(b->h_delay.begin() + (int64_t)c * S * NL, b->h_delay.begin() + (int64_t)(c + 1) * S * NL, dmin);
        int lane0 = 0;
        b->h_seg_off[c] = (int)b->h_segs.size();
        std::fill(lane_p.begin(), lane_p.end(), -1);
        for (int q : members[c]) {
            for (int j = 0; j < pcs[q].lanes; ++j) lane_p[lane0 + j] = q;
            b->h_segs.push_back(make_int4(pcs[q].row, lane0, lane0 + pcs[q].lanes, pcs[q].w));
            lane0 += pcs[q].lanes;
        }
        b->h_active[c] = lane0;
        assign_cells(b, c, lane_p, pcs, members[c], dmin);
        const int s0 = b->h_seg_off[c];
        const int ns = (int)b->h_segs.size() - s0;
        for (int w = 0; w < NW; ++w) {
            for (int sg = 0; sg < ns; ++sg) {
                const int4 g = b->h_segs[s0 + sg];
                if (g.z > w * 32 && g.y < w * 32 + 32) {
                    b->h_wfirst[c * NW + w] = sg;
                    break;
                }
            }
        }
    }
    b->h_seg_off[n_cta] = (int)b->h_segs.size();
    for (int64_t l = 0; l < b->F; ++l)
        if (b->slot_of_filter[l] < 0) return fail(SPIIR_EUNSUPPORTED, "internal: filter %lld was not placed", (long long)l);
    return SPIIR_OK;
}

static int upload(void **dst, const void *src, size_t bytes, const char *what) {
    SPIIR_TRY(dev_alloc(dst, bytes, what));
    if (bytes) SPIIR_CUDA_TRY(cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice));
    return SPIIR_OK;
}

static void bank_free_packed(spiir_bank_s *b) {
    dev_free(b->are); dev_free(b->aim); dev_free(b->bre); dev_free(b->bim);
    dev_free(b->dly); dev_free(b->state); dev_free(b->segs); dev_free(b->seg_off);
    dev_free(b->wfirst); dev_free(b->active); dev_free(b->win); dev_free(b->red_t); dev_free(b->red_off);
    dev_free(b->zpart);
    b->are = b->aim = b->bre = b->bim = nullptr;
    b->dly = nullptr;
    b->state = nullptr;
    b->segs = nullptr;
    b->seg_off = b->wfirst = b->active = nullptr;
    b->win = nullptr;
    b->red_t = b->red_off = nullptr;
    b->zpart = nullptr;
    b->zpart_pitch = 0;
}

static void bank_free(spiir_bank_s *b) {
    if (!b) return;
    int prev = -1;
    cudaGetDevice(&prev);
    if (b->device >= 0) cudaSetDevice(b->device);
    bank_free_packed(b);
    dev_free(b->xbuf[0]); dev_free(b->xbuf[1]);
    if (prev >= 0) cudaSetDevice(prev);
    delete b;
}

static int bank_alloc_device(spiir_bank_s *b) {
    SPIIR_TRY(upload((void **)&b->are, b->h_are.data(), b->h_are.size() * sizeof(float2), "a1.re"));
    SPIIR_TRY(upload((void **)&b->aim, b->h_aim.data(), b->h_aim.size() * sizeof(float2), "a1.im"));
    SPIIR_TRY(upload((void **)&b->bre, b->h_bre.data(), b->h_bre.size() * sizeof(float2), "b0.re"));
    SPIIR_TRY(upload((void **)&b->bim, b->h_bim.data(), b->h_bim.size() * sizeof(float2), "b0.im"));
    SPIIR_TRY(upload((void **)&b->dly, b->h_delay.data(), b->h_delay.size() * sizeof(int), "delays"));
    SPIIR_TRY(upload((void **)&b->segs, b->h_segs.data(), b->h_segs.size() * sizeof(int4), "segments"));
    SPIIR_TRY(upload((void **)&b->seg_off, b->h_seg_off.data(), b->h_seg_off.size() * sizeof(int), "segment offsets"));
    SPIIR_TRY(upload((void **)&b->wfirst, b->h_wfirst.data(), b->h_wfirst.size() * sizeof(int), "warp segments"));
    SPIIR_TRY(upload((void **)&b->active, b->h_active.data(), b->h_active.size() * sizeof(int), "active lanes"));
    SPIIR_TRY(upload((void **)&b->win, b->h_win.data(), b->h_win.size() * sizeof(int2), "block windows"));
    if (b->n_part > 0) {
        SPIIR_TRY(upload((void **)&b->red_t, b->h_red_t.data(), b->h_red_t.size() * sizeof(int), "split templates"));
        SPIIR_TRY(upload((void **)&b->red_off, b->h_red_off.data(), b->h_red_off.size() * sizeof(int), "piece offsets"));
    }
    b->state_det_stride = (int64_t)b->n_cta * (b->S / 2) * b->NL;
    SPIIR_TRY(dev_alloc((void **)&b->state, sizeof(float4) * b->state_det_stride * b->n_det, "IIR states"));
    SPIIR_CUDA_TRY(cudaMemset(b->state, 0, sizeof(float4) * b->state_det_stride * b->n_det));
    return SPIIR_OK;
}

// (Re)allocate the two strain windows for chunks of up to ncap samples, keeping history.
static int bank_reserve_zpart(spiir_bank_s *b, int64_t ncap) {
    if (b->n_part == 0 || (b->zpart && b->zpart_pitch >= ncap)) return SPIIR_OK;
    dev_free(b->zpart);
    b->zpart = nullptr;
    b->zpart_pitch = 0;
    SPIIR_TRY(dev_alloc((void **)&b->zpart, sizeof(float2) * ncap * b->n_det * b->n_part, "delay pieces"));
    b->zpart_pitch = ncap;
    return SPIIR_OK;
}

static int bank_reserve(spiir_bank_s *b, int64_t ncap, cudaStream_t stream) {
    SPIIR_TRY(bank_reserve_zpart(b, std::max(ncap, b->ncap)));
    if (ncap <= b->ncap && b->xbuf[0]) return SPIIR_OK;
    const int64_t pitch = ((b->D_pad + ncap + 3) / 4) * 4 + 4;
    float *nb[2] = {nullptr, nullptr};
    for (int i = 0; i < 2; ++i) {
        int rc = dev_alloc((void **)&nb[i], sizeof(float) * pitch * b->n_det, "strain window");
        if (rc != SPIIR_OK) {
            dev_free(nb[0]);
            return rc;
        }
        SPIIR_CUDA_TRY(cudaMemsetAsync(nb[i], 0, sizeof(float) * pitch * b->n_det, stream));
    }
    if (b->xbuf[0] && b->D_pad > 0)
        SPIIR_CUDA_TRY(cudaMemcpy2DAsync(nb[0], pitch * 4, b->xbuf[b->cur], b->xpitch * 4, b->D_pad * 4,
                                         b->n_det, cudaMemcpyDeviceToDevice, stream));
    SPIIR_CUDA_TRY(cudaStreamSynchronize(stream));
    dev_free(b->xbuf[0]);
    dev_free(b->xbuf[1]);
    b->xbuf[0] = nb[0];
    b->xbuf[1] = nb[1];
    b->cur = 0;
    b->xpitch = pitch;
    b->ncap = ncap;
    return SPIIR_OK;
}

int bank_prepare(spiir_bank_s *b, int64_t ncap, cudaStream_t stream) { return bank_reserve(b, ncap, stream); }

BankArgs bank_args(spiir_bank_s *b, float2 *z, int64_t zpitch, int64_t n) {
    BankArgs a{};
    a.xbuf = b->xbuf[b->cur];
    a.xpitch = b->xpitch;
    a.D_pad = b->D_pad;
    a.cta_win = b->win;
    a.n = n;
    a.c_tile = b->c_tile;
    a.are = b->are; a.aim = b->aim; a.bre = b->bre; a.bim = b->bim;
    a.delay = b->dly;
    a.state = b->state;
    a.state_det_stride = b->state_det_stride;
    a.segs = b->segs; a.seg_off = b->seg_off; a.wfirst = b->wfirst; a.cta_active = b->active;
    a.z = z;
    a.zpitch = zpitch;
    a.zpart = b->zpart;
    a.zpart_pitch = b->zpart_pitch;
    a.n_det = b->n_det;
    a.status = device_status_word();
    a.red_offset = bank_red_offset(b);
    a.n_cta_total = b->n_cta;
    a.n_pairs_total = (int64_t)b->n_cta * (b->S / 2) * b->NL;
    a.x_elems = b->xpitch * b->n_det;
    a.z_elems = INT64_MAX;
    a.n_segs_total = (int64_t)b->h_segs.size();
    a.zpart_elems = b->zpart_pitch * b->n_det * b->n_part;
    return a;
}

// z[t] += the later delay pieces of template t, added in bin order (deterministic).
__global__ void k_piece_sum(const int *red_t, const int *red_off, int n_det, const float2 *zpart, int64_t zpart_pitch,
                            float2 *z, int64_t zpitch, int64_t n) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int i = blockIdx.y / n_det, det = blockIdx.y % n_det;
    float2 *zp = z + ((int64_t)red_t[i] * n_det + det) * zpitch + k;
    float2 acc = *zp;
    for (int p = red_off[i]; p < red_off[i + 1]; ++p) {
        const float2 v = zpart[((int64_t)p * n_det + det) * zpart_pitch + k];
        acc.x += v.x;
        acc.y += v.y;
    }
    *zp = acc;
}

int bank_piece_sum(spiir_bank_s *b, float2 *z, int64_t zpitch, int64_t n, cudaStream_t stream) {
    const int n_red = (int)b->h_red_t.size();
    if (n_red == 0 || n < 1) return SPIIR_OK;
    if (n > b->zpart_pitch) return fail(SPIIR_EINVAL, "internal: %lld samples exceed the piece buffers", (long long)n);
    const dim3 grid((unsigned)((n + 255) / 256), (unsigned)(n_red * b->n_det));
    k_piece_sum<<<grid, 256, 0, stream>>>(b->red_t, b->red_off, b->n_det, b->zpart, b->zpart_pitch, z, zpitch, n);
    SPIIR_CUDA_TRY(cudaGetLastError());
    return SPIIR_OK;
}

template <int S, int NL, int R>
static int launch_persist(const PersistArgs &p, int blocks_per_sm, size_t smem, cudaStream_t s) {
    auto kern = k_filter_bank_persistent<S, NL, R>;
    cudaFuncAttributes fa{};
    SPIIR_CUDA_TRY(cudaFuncGetAttributes(&fa, kern));
    const int dyn_max = kBankMaxSmem - (int)fa.sharedSizeBytes;
    if ((int)smem > dyn_max) return fail(SPIIR_EUNSUPPORTED, "persistent filter kernel needs %zu bytes of shared memory", smem);
    SPIIR_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_max));
    int nb = 0, dev = 0, n_sm = 0;
    SPIIR_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, NL, smem));
    SPIIR_CUDA_TRY(cudaGetDevice(&dev));
    SPIIR_CUDA_TRY(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
    if (nb < 1) return fail(SPIIR_EUNSUPPORTED, "persistent filter kernel does not fit on an SM");
    const int per_sm = blocks_per_sm > 0 ? std::min(blocks_per_sm, nb) : nb;
    const int grid = std::max(1, std::min(p.n_items, n_sm * per_sm));
    kern<<<grid, NL, smem, s>>>(p);
    SPIIR_CUDA_TRY(cudaGetLastError());
    return SPIIR_OK;
}

int bank_launch_persistent(const PersistArgs &p, int S, int NL, int R, int blocks_per_sm, size_t smem,
                           cudaStream_t s) {
#define SPIIR_PERSIST(S_, NL_, R_) \
    if (S == S_ && NL == NL_ && R == R_) return launch_persist<S_, NL_, R_>(p, blocks_per_sm, smem, s);
    SPIIR_PERSIST(8, 128, 32) SPIIR_PERSIST(8, 256, 32) SPIIR_PERSIST(8, 128, 16) SPIIR_PERSIST(8, 256, 16)
    SPIIR_PERSIST(16, 128, 32) SPIIR_PERSIST(16, 256, 32) SPIIR_PERSIST(16, 128, 16) SPIIR_PERSIST(16, 256, 16)
    SPIIR_PERSIST(4, 128, 32) SPIIR_PERSIST(4, 256, 32) SPIIR_PERSIST(4, 128, 16) SPIIR_PERSIST(4, 256, 16)
#undef SPIIR_PERSIST
    return fail(SPIIR_EINVAL, "unsupported persistent shape");
}

int bank_filter(spiir_bank_s *b, const float *strain, int64_t strain_pitch, int64_t n, float2 *z,
                int64_t zpitch, cudaStream_t stream) {
    SPIIR_TRY(bank_reserve(b, std::max<int64_t>(n, 2048), stream));
    float *x = b->xbuf[b->cur];
    SPIIR_CUDA_TRY(cudaMemcpy2DAsync(x + b->D_pad, b->xpitch * 4, strain, strain_pitch * 4, n * 4, b->n_det,
                                     cudaMemcpyDeviceToDevice, stream));
    const BankArgs a = bank_args(b, z, zpitch, n);
    const size_t smem = bank_smem_bytes(b);
    if (smem > (size_t)kBankMaxSmem)
        return fail(SPIIR_EUNSUPPORTED, "strain window of %d + %d samples does not fit in shared memory",
                    b->win_max, b->c_tile);
    SPIIR_TRY(launch_bank_any(b, a, smem, stream));
    SPIIR_TRY(bank_piece_sum(b, z, zpitch, n, stream));
    // the last D_pad samples become the history of the next call
    const int nxt = 1 - b->cur;
    if (b->D_pad > 0)
        SPIIR_CUDA_TRY(cudaMemcpy2DAsync(b->xbuf[nxt], b->xpitch * 4, x + n, b->xpitch * 4, b->D_pad * 4,
                                         b->n_det, cudaMemcpyDeviceToDevice, stream));
    b->cur = nxt;
    return SPIIR_OK;
}

}  // namespace spiir

using namespace spiir;

// ---------------------------------------------------------------------------------------
// C ABI

extern "C" int spiir_bank_create(int n_det, int n_templates, const int64_t *off, const float *a1,
                                 const float *b0, const int32_t *delay, spiir_bank_t *out) {
    clear_error();
    if (!out) return fail(SPIIR_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_det < 1 || n_det > 8) return fail(SPIIR_EINVAL, "n_det = %d outside [1, 8]", n_det);
    if (n_templates < 1) return fail(SPIIR_EINVAL, "n_templates = %d < 1", n_templates);
    if (!off) return fail(SPIIR_EINVAL, "filter_offsets is NULL");
    if (off[0] != 0) return fail(SPIIR_EINVAL, "filter_offsets[0] = %lld, expected 0", (long long)off[0]);
    for (int t = 0; t < n_templates; ++t)
        if (off[t + 1] < off[t]) return fail(SPIIR_EINVAL, "filter_offsets decrease at template %d", t);
    const int64_t F = off[n_templates];
    if (F > 0 && (!a1 || !b0 || !delay)) return fail(SPIIR_EINVAL, "coefficient pointer is NULL");
    int32_t dmax = 0;
    for (int64_t l = 0; l < F; ++l) {
        const double ar = a1[2 * l], ai = a1[2 * l + 1], br = b0[2 * l], bi = b0[2 * l + 1];
        if (!std::isfinite(ar) || !std::isfinite(ai) || !std::isfinite(br) || !std::isfinite(bi))
            return fail(SPIIR_EINVAL, "filter %lld has a non-finite coefficient", (long long)l);
        if (ar * ar + ai * ai >= 1.0)
            return fail(SPIIR_EINVAL, "filter %lld has |a1| >= 1 (unstable)", (long long)l);
        if (delay[l] < 0 || delay[l] > kBankMaxDelay)
            return fail(SPIIR_EINVAL, "filter %lld has delay %d outside [0, %d]", (long long)l, delay[l],
                        kBankMaxDelay);
        dmax = std::max(dmax, delay[l]);
    }
    spiir_bank_s *b = new (std::nothrow) spiir_bank_s();
    if (!b) return fail(SPIIR_ENOMEM, "host allocation of the bank failed");
    cudaGetDevice(&b->device);
    b->n_det = n_det;
    b->T = n_templates;
    b->F = F;
    b->dmax = dmax;
    b->D_pad = ((dmax + 3) / 4) * 4;
    b->offsets.assign(off, off + n_templates + 1);
    b->a1.assign(a1, a1 + 2 * F);
    b->b0.assign(b0, b0 + 2 * F);
    b->delay.assign(delay, delay + F);
    int64_t fmax = 0;
    for (int t = 0; t < n_templates; ++t) fmax = std::max(fmax, off[t + 1] - off[t]);
    // default launch shape (fastest measured on the online-sized bank): 8 filters per lane,
    // 128 lanes per block; larger blocks, then 16 filters per lane, for big templates
    b->S = 8;
    b->NL = 128;
    b->R = 32;
    if (fmax > (int64_t)b->S * b->NL) b->NL = 256;
    if (fmax > (int64_t)b->S * b->NL) b->S = 16;
    b->c_tile = kBankTile;
    // long delays: blocks hold one delay bin each, so that every block's strain window stays
    // within the bin width plus the tile
    b->dbin = dmax >= kBankSplitDelay ? kBankDefaultBin : 0;
    if (b->dbin > 0 && b->S == 8) b->NL = 256;
    int rc = bank_pack(b);
    if (rc == SPIIR_OK) {
        const size_t smem = bank_smem_bytes(b);
        if (smem > (size_t)kBankMaxSmem)
            rc = fail(SPIIR_EUNSUPPORTED, "a block's delay span %d needs a %zu-byte window; limit %d", b->win_max,
                      smem, kBankMaxSmem);
    }
    if (rc == SPIIR_OK) rc = bank_alloc_device(b);
    if (rc == SPIIR_OK) rc = bank_reserve(b, 2048, 0);
    if (rc != SPIIR_OK) {
        bank_free(b);
        return rc;
    }
    *out = b;
    return SPIIR_OK;
}

extern "C" void spiir_bank_destroy(spiir_bank_t b) { bank_free(b); }

extern "C" int spiir_bank_info(spiir_bank_t b, int *n_det, int *n_templates, int64_t *n_filters,
                               int32_t *max_delay) {
    if (!b) return fail(SPIIR_EINVAL, "bank is NULL");
    if (n_det) *n_det = b->n_det;
    if (n_templates) *n_templates = b->T;
    if (n_filters) *n_filters = b->F;
    if (max_delay) *max_delay = b->dmax;
    return SPIIR_OK;
}

extern "C" int spiir_bank_reset(spiir_bank_t b, void *stream) {
    if (!b) return fail(SPIIR_EINVAL, "bank is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    SPIIR_CUDA_TRY(cudaMemsetAsync(b->state, 0, sizeof(float4) * b->state_det_stride * b->n_det, s));
    for (int i = 0; i < 2; ++i)
        if (b->xbuf[i]) SPIIR_CUDA_TRY(cudaMemsetAsync(b->xbuf[i], 0, sizeof(float) * b->xpitch * b->n_det, s));
    return SPIIR_OK;
}

extern "C" int spiir_bank_state_bytes(spiir_bank_t b, size_t *bytes) {
    if (!b || !bytes) return fail(SPIIR_EINVAL, "NULL argument");
    *bytes = (size_t)b->n_det * b->F * 2 * sizeof(float) + (size_t)b->n_det * b->dmax * sizeof(float);
    return SPIIR_OK;
}

extern "C" int spiir_bank_get_state(spiir_bank_t b, void *host, size_t bytes) {
    size_t need = 0;
    SPIIR_TRY(spiir_bank_state_bytes(b, &need));
    if (!host || bytes != need) return fail(SPIIR_EINVAL, "state buffer has %zu bytes, need %zu", bytes, need);
    SPIIR_CUDA_TRY(cudaDeviceSynchronize());
    std::vector<float4> st((size_t)b->state_det_stride * b->n_det);
    SPIIR_CUDA_TRY(cudaMemcpy(st.data(), b->state, st.size() * sizeof(float4), cudaMemcpyDeviceToHost));
    float *o = static_cast<float *>(host);
    const int NP = b->S / 2;
    for (int d = 0; d < b->n_det; ++d)
        for (int64_t l = 0; l < b->F; ++l) {
            const int64_t slot = b->slot_of_filter[l];
            const int64_t ln = slot % b->NL, cs = slot / b->NL, s = cs % b->S, c = cs / b->S;
            const float4 v = st[(size_t)d * b->state_det_stride + ((size_t)c * NP + s / 2) * b->NL + ln];
            o[((size_t)d * b->F + l) * 2] = (s % 2 == 0) ? v.x : v.y;
            o[((size_t)d * b->F + l) * 2 + 1] = (s % 2 == 0) ? v.z : v.w;
        }
    float *h = o + (size_t)b->n_det * b->F * 2;
    if (b->dmax > 0)
        SPIIR_CUDA_TRY(cudaMemcpy2D(h, b->dmax * 4, b->xbuf[b->cur] + (b->D_pad - b->dmax), b->xpitch * 4,
                                    b->dmax * 4, b->n_det, cudaMemcpyDeviceToHost));
    return SPIIR_OK;
}

extern "C" int spiir_bank_set_state(spiir_bank_t b, const void *host, size_t bytes) {
    size_t need = 0;
    SPIIR_TRY(spiir_bank_state_bytes(b, &need));
    if (!host || bytes != need) return fail(SPIIR_EINVAL, "state buffer has %zu bytes, need %zu", bytes, need);
    const float *in = static_cast<const float *>(host);
    for (size_t i = 0; i < need / sizeof(float); ++i)
        if (!std::isfinite(in[i])) return fail(SPIIR_EINVAL, "state holds a non-finite value at %zu", i);
    SPIIR_CUDA_TRY(cudaDeviceSynchronize());
    std::vector<float4> st((size_t)b->state_det_stride * b->n_det, make_float4(0, 0, 0, 0));
    const int NP = b->S / 2;
    for (int d = 0; d < b->n_det; ++d)
        for (int64_t l = 0; l < b->F; ++l) {
            const int64_t slot = b->slot_of_filter[l];
            const int64_t ln = slot % b->NL, cs = slot / b->NL, s = cs % b->S, c = cs / b->S;
            float4 &v = st[(size_t)d * b->state_det_stride + ((size_t)c * NP + s / 2) * b->NL + ln];
            const float re = in[((size_t)d * b->F + l) * 2], im = in[((size_t)d * b->F + l) * 2 + 1];
            if (s % 2 == 0) { v.x = re; v.z = im; } else { v.y = re; v.w = im; }
        }
    SPIIR_CUDA_TRY(cudaMemcpy(b->state, st.data(), st.size() * sizeof(float4), cudaMemcpyHostToDevice));
    for (int i = 0; i < 2; ++i)
        SPIIR_CUDA_TRY(cudaMemset(b->xbuf[i], 0, sizeof(float) * b->xpitch * b->n_det));
    const float *h = in + (size_t)b->n_det * b->F * 2;
    if (b->dmax > 0)
        SPIIR_CUDA_TRY(cudaMemcpy2D(b->xbuf[b->cur] + (b->D_pad - b->dmax), b->xpitch * 4, h, b->dmax * 4,
                                    b->dmax * 4, b->n_det, cudaMemcpyHostToDevice));
    return SPIIR_OK;
}

extern "C" int spiir_filter_chunk(spiir_bank_t b, const float *strain, int64_t strain_pitch, int64_t n,
                                  float *snr, int64_t snr_pitch, void *stream) {
    clear_error();
    if (!b) return fail(SPIIR_EINVAL, "bank is NULL");
    if (!strain || !snr) return fail(SPIIR_EINVAL, "strain or snr pointer is NULL");
    if (n < 1) return fail(SPIIR_EINVAL, "n = %lld < 1", (long long)n);
    if (strain_pitch < n || snr_pitch < n)
        return fail(SPIIR_EINVAL, "pitch smaller than n (strain %lld, snr %lld, n %lld)", (long long)strain_pitch,
                    (long long)snr_pitch, (long long)n);
    if (((uintptr_t)snr) % 8 != 0) return fail(SPIIR_EINVAL, "snr pointer is not 8-byte aligned");
    return bank_filter(b, strain, strain_pitch, n, reinterpret_cast<float2 *>(snr), snr_pitch,
                       (cudaStream_t)stream);
}

// Re-pack the bank for a new launch shape or delay-bin width, keeping the streaming state.  On
// failure the previous shape is restored and the bank stays usable.
static int bank_repack(spiir_bank_s *b, int S, int NL, int R, int tile, int dbin) {
    size_t nb = 0;
    SPIIR_TRY(spiir_bank_state_bytes(b, &nb));
    std::vector<char> saved(nb);
    SPIIR_TRY(spiir_bank_get_state(b, saved.data(), nb));
    const int oS = b->S, oNL = b->NL, oR = b->R, oT = b->c_tile, oB = b->dbin;
    b->S = S;
    b->NL = NL;
    b->R = R;
    b->c_tile = tile;
    b->dbin = dbin;
    bank_free_packed(b);
    int rc = bank_pack(b);
    if (rc == SPIIR_OK && bank_smem_bytes(b) > (size_t)kBankMaxSmem)
        rc = fail(SPIIR_EUNSUPPORTED, "shape needs %zu bytes of shared memory (window span %d + tile %d)",
                  bank_smem_bytes(b), b->win_max, tile);
    if (rc == SPIIR_OK) rc = bank_alloc_device(b);
    if (rc == SPIIR_OK) rc = bank_reserve_zpart(b, b->ncap);
    if (rc == SPIIR_OK) rc = spiir_bank_set_state(b, saved.data(), nb);
    if (rc != SPIIR_OK) {
        const std::string msg = [] { char m[512]; spiir_last_error(m, sizeof m); return std::string(m); }();
        bank_free_packed(b);
        b->S = oS; b->NL = oNL; b->R = oR; b->c_tile = oT; b->dbin = oB;
        if (bank_pack(b) == SPIIR_OK && bank_alloc_device(b) == SPIIR_OK && bank_reserve_zpart(b, b->ncap) == SPIIR_OK)
            spiir_bank_set_state(b, saved.data(), nb);
        return fail(rc, "%s", msg.c_str());
    }
    return SPIIR_OK;
}

extern "C" int spiir_bank_set_shape(spiir_bank_t b, int filters_per_lane, int lanes_per_block, int steps_per_reduce,
                                    int tile) {
    clear_error();
    if (!b) return fail(SPIIR_EINVAL, "bank is NULL");
    if (filters_per_lane != 4 && filters_per_lane != 8 && filters_per_lane != 16)
        return fail(SPIIR_EINVAL, "filters_per_lane must be 4, 8 or 16");
    if (lanes_per_block != 128 && lanes_per_block != 256) return fail(SPIIR_EINVAL, "lanes_per_block must be 128 or 256");
    if (steps_per_reduce != 16 && steps_per_reduce != 20 && steps_per_reduce != 32 && steps_per_reduce != 64)
        return fail(SPIIR_EINVAL, "steps_per_reduce must be 16, 20, 32 or 64");
    if (tile < steps_per_reduce || tile > 8192 || tile % steps_per_reduce != 0)
        return fail(SPIIR_EINVAL, "tile must be a multiple of steps_per_reduce in [steps_per_reduce, 8192]");
    int64_t fmax = 0;
    for (int t = 0; t < b->T; ++t) fmax = std::max(fmax, b->offsets[t + 1] - b->offsets[t]);
    if (fmax > (int64_t)filters_per_lane * lanes_per_block)
        return fail(SPIIR_EUNSUPPORTED, "a template has %lld filters, more than %d lanes x %d", (long long)fmax,
                    lanes_per_block, filters_per_lane);
    return bank_repack(b, filters_per_lane, lanes_per_block, steps_per_reduce, tile, b->dbin);
}

extern "C" int spiir_bank_set_delay_bin(spiir_bank_t b, int32_t delay_bin) {
    clear_error();
    if (!b) return fail(SPIIR_EINVAL, "bank is NULL");
    if (delay_bin != 0 && (delay_bin < 1024 || delay_bin > kBankMaxDelay || delay_bin % 4 != 0))
        return fail(SPIIR_EINVAL, "delay_bin %d must be 0 or a multiple of 4 in [1024, %d]", delay_bin, kBankMaxDelay);
    return bank_repack(b, b->S, b->NL, b->R, b->c_tile, delay_bin);
}

extern "C" int spiir_bank_get_delay_bin(spiir_bank_t b, int32_t *delay_bin, int *n_blocks, int *n_pieces) {
    if (!b) return fail(SPIIR_EINVAL, "bank is NULL");
    if (delay_bin) *delay_bin = b->dbin;
    if (n_blocks) *n_blocks = b->n_cta;
    if (n_pieces) *n_pieces = b->T + b->n_part;
    return SPIIR_OK;
}

extern "C" int spiir_bank_get_shape(spiir_bank_t b, int *filters_per_lane, int *lanes_per_block,
                                    int *steps_per_reduce, int *tile) {
    if (!b) return fail(SPIIR_EINVAL, "bank is NULL");
    if (filters_per_lane) *filters_per_lane = b->S;
    if (lanes_per_block) *lanes_per_block = b->NL;
    if (steps_per_reduce) *steps_per_reduce = b->R;
    if (tile) *tile = b->c_tile;
    return SPIIR_OK;
}

// ---------------------------------------------------------------------------------------
// Filter bank without any allocation (spiir_filter_static).
//
// Some callers cannot allocate device memory: code that runs where cudaMalloc is not
// allowed or would stall (inside a real-time loop, under an allocator that owns all device
// memory, or in a process that must not grow its footprint after start-up).  This entry
// point runs the same filter-bank kernel as spiir_filter_chunk on one segment that starts a
// stream (zero IIR states, zero strain history), with every piece of scratch -- the copied
// coefficients, their packed layout, the block tables, the IIR states and the strain window
// -- carved out of one file-scope device array of fixed size.  The array exists on every GPU
// that loads the library, for the life of the process.  All calls share it, so calls whose
// GPU work overlaps (different streams, no ordering) race and corrupt each other's results.
// A bounded wait that runs out is recorded in the library's status word (itself a file-scope
// device variable), which spiir_device_status reports.

namespace spiir {

constexpr size_t kStaticScratchBytes = size_t(32) << 20;  // 32 MiB
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Device address of the scratch array in the current device's context.  In host code the
// array's name is only a host-side stand-in, so the address is looked up with the device
// current -- on every call, which is cheap once the module is loaded and stays right after
// the context has been re-created.
static int static_scratch_address(unsigned char **out) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return fail(SPIIR_ECUDA, "cudaGetSymbolAddress of the static scratch failed: %s", cudaGetErrorString(e));
    }
    *out = static_cast<unsigned char *>(p);
    return SPIIR_OK;
}

// Block layout in template order: template t takes max(1, ceil(F_t / S)) lanes; a block is
// closed when the next template does not fit.  One thread; T is small.
__global__ void k_static_layout(const int64_t *off, int T, int S, int NL, int D_pad, int *cta_of_t, int *lane0_of_t,
                                int4 *segs, int *seg_off, int *wfirst, int *active, int2 *win) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int NW = NL / 32;
    int c = 0, used = 0;
    seg_off[0] = 0;
    for (int t = 0; t < T; ++t) {
        const int64_t f = off[t + 1] - off[t];
        const int L = (int)max((int64_t)1, (f + S - 1) / S);
        if (used + L > NL) {
            active[c] = used;
            ++c;
            used = 0;
            seg_off[c] = t;
        }
        cta_of_t[t] = c;
        lane0_of_t[t] = used;
        segs[t] = make_int4(t, used, used + L, 0);
        used += L;
    }
    active[c] = used;
    seg_off[c + 1] = T;
    for (int cc = 0; cc <= c; ++cc) {
        win[cc] = make_int2(D_pad, D_pad);  // every block stages the whole history
        const int s0 = seg_off[cc], ns = seg_off[cc + 1] - s0;
        for (int w = 0; w < NW; ++w) {
            int first = -1;
            for (int sg = 0; sg < ns; ++sg) {
                const int4 g = segs[s0 + sg];
                if (g.z > w * 32 && g.y < w * 32 + 32) {
                    first = sg;
                    break;
                }
            }
            wfirst[cc * NW + w] = first;
        }
    }
}

// Scatter filter l of template t to lane lane0[t] + q / S, slot q % S (q = l - off[t]).
__global__ void k_static_scatter(const int64_t *off, const float2 *a1, const float2 *b0, const int32_t *delay, int T,
                                 int64_t F, int S, int NL, const int *cta_of_t, const int *lane0_of_t, float2 *are,
                                 float2 *aim, float2 *bre, float2 *bim, int *dly) {
    const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= F) return;
    int lo = 0, hi = T;  // last t with off[t] <= l
    while (hi - lo > 1) {
        const int mid = (lo + hi) / 2;
        if (off[mid] <= l) lo = mid; else hi = mid;
    }
    const int t = lo;
    const int64_t q = l - off[t];
    const int lane = lane0_of_t[t] + (int)(q / S), s = (int)(q % S), c = cta_of_t[t];
    const int NP = S / 2;
    const int64_t pi = ((int64_t)c * NP + s / 2) * NL + lane;
    float *ar = reinterpret_cast<float *>(&are[pi]) + (s & 1);
    float *ai = reinterpret_cast<float *>(&aim[pi]) + (s & 1);
    float *br = reinterpret_cast<float *>(&bre[pi]) + (s & 1);
    float *bi = reinterpret_cast<float *>(&bim[pi]) + (s & 1);
    *ar = a1[l].x;
    *ai = a1[l].y;
    *br = b0[l].x;
    *bi = b0[l].y;
    dly[((int64_t)c * S + s) * NL + lane] = delay[l];
}

}  // namespace spiir

extern "C" int spiir_filter_static(int n_det, int n_templates, const int64_t *off, const float *a1, const float *b0,
                                   const int32_t *delay, const float *strain, int64_t strain_pitch, int64_t n,
                                   float *snr, int64_t snr_pitch, void *stream) {
    clear_error();
    cudaStream_t st = (cudaStream_t)stream;
    // host-side validation (reads the caller's host arrays only)
    if (n_det < 1 || n_det > kStaticMaxDet) return fail(SPIIR_EINVAL, "n_det = %d outside [1, %d]", n_det, kStaticMaxDet);
    if (n_templates < 1) return fail(SPIIR_EINVAL, "n_templates = %d < 1", n_templates);
    if (!off || !strain || !snr) return fail(SPIIR_EINVAL, "NULL pointer");
    if (off[0] != 0) return fail(SPIIR_EINVAL, "filter_offsets[0] must be 0");
    if (n < 1 || strain_pitch < n || snr_pitch < n) return fail(SPIIR_EINVAL, "bad n or pitch");
    if (((uintptr_t)snr) % 8 != 0) return fail(SPIIR_EINVAL, "snr pointer is not 8-byte aligned");
    int64_t fmax = 0;
    for (int t = 0; t < n_templates; ++t) {
        if (off[t + 1] < off[t]) return fail(SPIIR_EINVAL, "filter_offsets decrease at template %d", t);
        fmax = std::max(fmax, off[t + 1] - off[t]);
    }
    const int64_t F = off[n_templates];
    if (F > 0 && (!a1 || !b0 || !delay)) return fail(SPIIR_EINVAL, "coefficient pointer is NULL");
    if (n_templates > kStaticMaxTemplates || F > kStaticMaxFilters || n > kStaticMaxSamples)
        return fail(SPIIR_EUNSUPPORTED,
                    "static scratch limits: at most %d templates, %d filters, %d samples (got %d, %lld, %lld)",
                    kStaticMaxTemplates, kStaticMaxFilters, kStaticMaxSamples, n_templates, (long long)F, (long long)n);
    int32_t dmax = 0;
    for (int64_t l = 0; l < F; ++l) {
        const double ar = a1[2 * l], ai = a1[2 * l + 1], br = b0[2 * l], bi = b0[2 * l + 1];
        if (!std::isfinite(ar) || !std::isfinite(ai) || !std::isfinite(br) || !std::isfinite(bi))
            return fail(SPIIR_EINVAL, "filter %lld has a non-finite coefficient", (long long)l);
        if (ar * ar + ai * ai >= 1.0) return fail(SPIIR_EINVAL, "filter %lld has |a1| >= 1 (unstable)", (long long)l);
        if (delay[l] < 0 || delay[l] > kStaticMaxDelay)
            return fail(SPIIR_EINVAL, "filter %lld has delay %d outside [0, %d]", (long long)l, delay[l], kStaticMaxDelay);
        dmax = std::max(dmax, delay[l]);
    }
    // launch shape as the allocating path chooses it for a new bank
    const int S = fmax > 2048 ? 16 : 8;
    const int NL = fmax > 1024 ? 256 : 128;
    const int R = 32, tile = kBankTile, NP = S / 2;
    if (fmax > (int64_t)S * NL) return fail(SPIIR_EUNSUPPORTED, "a template has %lld filters", (long long)fmax);
    int n_cta = 1, used = 0;
    for (int t = 0; t < n_templates; ++t) {
        const int L = (int)std::max<int64_t>(1, (off[t + 1] - off[t] + S - 1) / S);
        if (used + L > NL) {
            ++n_cta;
            used = 0;
        }
        used += L;
    }
    const int D_pad = ((dmax + 3) / 4) * 4;
    const int64_t xpitch = ((D_pad + n + 3) / 4) * 4 + 4;
    // carve the scratch
    size_t cur = 0;
    auto take = [&](size_t bytes) {
        const size_t at = cur;
        cur = (cur + bytes + 255) / 256 * 256;
        return at;
    };
    const int64_t npair = (int64_t)n_cta * NP * NL;
    const size_t o_off = take(sizeof(int64_t) * (n_templates + 1));
    const size_t o_a1 = take(sizeof(float2) * F), o_b0 = take(sizeof(float2) * F), o_d = take(sizeof(int32_t) * F);
    const size_t o_pk = cur;
    const size_t o_are = take(sizeof(float2) * npair), o_aim = take(sizeof(float2) * npair);
    const size_t o_bre = take(sizeof(float2) * npair), o_bim = take(sizeof(float2) * npair);
    const size_t o_dly = take(sizeof(int) * npair * 2);
    const size_t o_st = take(sizeof(float4) * npair * n_det);
    const size_t pk_bytes = cur - o_pk;
    const size_t o_cta = take(sizeof(int) * n_templates), o_l0 = take(sizeof(int) * n_templates);
    const size_t o_segs = take(sizeof(int4) * n_templates), o_so = take(sizeof(int) * (n_cta + 1));
    const size_t o_wf = take(sizeof(int) * n_cta * (NL / 32)), o_act = take(sizeof(int) * n_cta);
    const size_t o_win = take(sizeof(int2) * n_cta);
    const size_t o_x = take(sizeof(float) * xpitch * n_det);
    if (cur > kStaticScratchBytes)
        return fail(SPIIR_EUNSUPPORTED, "problem needs %zu bytes of scratch; the static array holds %zu", cur,
                    kStaticScratchBytes);
    BankArgs a{};
    a.red_offset = kBankSmemHead + (size_t)(((D_pad + tile + 3) / 4) * 4 * sizeof(float) + 127) / 128 * 128;
    const size_t smem = a.red_offset + (size_t)NL * bank_red_stride(R) * sizeof(float2);
    if (smem > (size_t)kBankMaxSmem) return fail(SPIIR_EUNSUPPORTED, "strain window does not fit in shared memory");
    unsigned char *base = nullptr;
    SPIIR_TRY(static_scratch_address(&base));
    int *status = device_status_word();
    if (!status) return fail(SPIIR_ECUDA, "device status word unavailable");
    // inputs into the scratch, packed region and strain window cleared
    SPIIR_CUDA_TRY(cudaMemcpyAsync(base + o_off, off, sizeof(int64_t) * (n_templates + 1), cudaMemcpyHostToDevice, st));
    if (F > 0) {
        SPIIR_CUDA_TRY(cudaMemcpyAsync(base + o_a1, a1, sizeof(float2) * F, cudaMemcpyHostToDevice, st));
        SPIIR_CUDA_TRY(cudaMemcpyAsync(base + o_b0, b0, sizeof(float2) * F, cudaMemcpyHostToDevice, st));
        SPIIR_CUDA_TRY(cudaMemcpyAsync(base + o_d, delay, sizeof(int32_t) * F, cudaMemcpyHostToDevice, st));
    }
    SPIIR_CUDA_TRY(cudaMemsetAsync(base + o_pk, 0, pk_bytes, st));
    SPIIR_CUDA_TRY(cudaMemsetAsync(base + o_x, 0, sizeof(float) * xpitch * n_det, st));
    SPIIR_CUDA_TRY(cudaMemcpy2DAsync(reinterpret_cast<float *>(base + o_x) + D_pad, xpitch * sizeof(float), strain,
                                     strain_pitch * sizeof(float), n * sizeof(float), n_det, cudaMemcpyDeviceToDevice,
                                     st));
    k_static_layout<<<1, 32, 0, st>>>(reinterpret_cast<const int64_t *>(base + o_off), n_templates, S, NL, D_pad,
                                      reinterpret_cast<int *>(base + o_cta), reinterpret_cast<int *>(base + o_l0),
                                      reinterpret_cast<int4 *>(base + o_segs), reinterpret_cast<int *>(base + o_so),
                                      reinterpret_cast<int *>(base + o_wf), reinterpret_cast<int *>(base + o_act),
                                      reinterpret_cast<int2 *>(base + o_win));
    SPIIR_CUDA_TRY(cudaGetLastError());
    if (F > 0) {
        const int nb = (int)((F + 255) / 256);
        k_static_scatter<<<nb, 256, 0, st>>>(
            reinterpret_cast<const int64_t *>(base + o_off), reinterpret_cast<const float2 *>(base + o_a1),
            reinterpret_cast<const float2 *>(base + o_b0), reinterpret_cast<const int32_t *>(base + o_d), n_templates, F,
            S, NL, reinterpret_cast<const int *>(base + o_cta), reinterpret_cast<const int *>(base + o_l0),
            reinterpret_cast<float2 *>(base + o_are), reinterpret_cast<float2 *>(base + o_aim),
            reinterpret_cast<float2 *>(base + o_bre), reinterpret_cast<float2 *>(base + o_bim),
            reinterpret_cast<int *>(base + o_dly));
        SPIIR_CUDA_TRY(cudaGetLastError());
    }
    a.xbuf = reinterpret_cast<const float *>(base + o_x);
    a.xpitch = xpitch;
    a.D_pad = D_pad;
    a.cta_win = reinterpret_cast<const int2 *>(base + o_win);
    a.n = n;
    a.c_tile = tile;
    a.are = reinterpret_cast<const float2 *>(base + o_are);
    a.aim = reinterpret_cast<const float2 *>(base + o_aim);
    a.bre = reinterpret_cast<const float2 *>(base + o_bre);
    a.bim = reinterpret_cast<const float2 *>(base + o_bim);
    a.delay = reinterpret_cast<const int *>(base + o_dly);
    a.state = reinterpret_cast<float4 *>(base + o_st);
    a.state_det_stride = npair;
    a.segs = reinterpret_cast<const int4 *>(base + o_segs);
    a.seg_off = reinterpret_cast<const int *>(base + o_so);
    a.wfirst = reinterpret_cast<const int *>(base + o_wf);
    a.cta_active = reinterpret_cast<const int *>(base + o_act);
    a.z = reinterpret_cast<float2 *>(snr);
    a.zpitch = snr_pitch;
    a.n_det = n_det;
    a.status = status;
    a.n_cta_total = n_cta;
    a.n_pairs_total = npair;
    a.x_elems = xpitch * n_det;
    a.z_elems = INT64_MAX;
    a.n_segs_total = n_templates;
    if (S == 8) return launch_bank_nl<8>(a, NL, R, n_cta, n_det, smem, st);
    return launch_bank_nl<16>(a, NL, R, n_cta, n_det, smem, st);
}
