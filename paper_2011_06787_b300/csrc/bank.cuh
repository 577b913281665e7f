// Filter-bank object and kernel arguments (internal).
#pragma once

#include <vector>

#include "common.cuh"

namespace spiir {

constexpr int kBankTile = 1024;                // default time steps per staged strain window
constexpr int kBankSmemHead = 128;             // bytes before the strain window (mbarrier)
constexpr int kMaxBands = 4;                   // banks per persistent launch
constexpr int kBankMaxSmem = 227 * 1024;       // dynamic shared memory limit per block
constexpr int kBankMaxDelay = 1 << 20;         // largest delay (samples)
// Banks whose largest delay reaches kBankSplitDelay are cut into delay bins of kBankDefaultBin
// samples: a block holds the filters of one bin only and stages that bin's window.  Such banks
// default to 256-lane blocks (fewer pieces per block boundary, two blocks of eight warps per SM
// with the larger windows): on 4096 whole chirps from 30 Hz x 600 filters, bins of 8192 with
// 256 lanes measured 7.06 ms per 1 s chunk against 7.72 ms for bins of 16384 with 128 lanes.
constexpr int kBankSplitDelay = 16384;
constexpr int kBankDefaultBin = 8192;
// limits of spiir_filter_static (fixed-size static scratch)
constexpr int kStaticMaxDet = 4;
constexpr int kStaticMaxTemplates = 4096;
constexpr int kStaticMaxFilters = 131072;
constexpr int kStaticMaxSamples = 65536;
constexpr int kStaticMaxDelay = 8192;

struct BankArgs {
    const float *xbuf;        // [n_det][xpitch] window source: D_pad history + chunk
    int64_t xpitch;
    int D_pad;                // history length (>= max delay, multiple of 4)
    const int2 *cta_win;      // [n_cta] (dhi, span): block c stages x[k0 - dhi, k0 - dhi + span + tile)
    int64_t n;                // samples in this call
    int c_tile;               // samples per staged window
    const float2 *are, *aim, *bre, *bim;  // [n_cta][S/2][NL] packed pairs of filters
    const int *delay;         // [n_cta][S][NL]
    float4 *state;            // [n_det][n_cta][S/2][NL] (re0, re1, im0, im1)
    int64_t state_det_stride;
    const int4 *segs;         // (template, lane_lo, lane_hi, 0) per template, grouped by block
    const int *seg_off;       // [n_cta + 1]
    const int *wfirst;        // [n_cta][warps] first block-local segment touching each warp, -1 none
    const int *cta_active;    // [n_cta] lanes in use
    float2 *z;                // [T][n_det][zpitch]
    int64_t zpitch;
    float2 *zpart;            // [n_part][n_det][zpart_pitch]: later delay pieces of split templates
    int64_t zpart_pitch;
    int n_det;
    int *status;
    size_t red_offset;        // byte offset of the reduction buffer in shared memory
    // buffer sizes, used by the bounds-checked debug build (SPIIR_CHECKED)
    int n_cta_total;
    int64_t n_pairs_total, x_elems, z_elems, n_segs_total, zpart_elems;
};

struct PersistArgs {
    BankArgs banks[kMaxBands];
    const int4 *items;        // (bank, block, detector, 0), in the order blocks take them
    int n_items;
    int *counter;             // zero before the launch
};

}  // namespace spiir

struct spiir_bank_s {
    int device = -1;
    int n_det = 0, T = 0;
    int64_t F = 0;
    int32_t dmax = 0;
    int D_pad = 0;
    int S = 8;        // filters per lane
    int NL = 256;     // lanes (threads) per block
    int R = 32;       // time steps per reduction block
    int c_tile = 1024;
    int dbin = 0;     // delay-bin width (0: one bin); see kBankSplitDelay
    int n_cta = 0;
    int win_max = 0;  // largest block window span (samples)
    int n_part = 0;   // zpart rows: second and later delay pieces of split templates
    std::vector<int64_t> offsets;
    std::vector<float> a1, b0;
    std::vector<int32_t> delay;
    // packed host images
    std::vector<float2> h_are, h_aim, h_bre, h_bim;
    std::vector<int> h_delay;
    std::vector<int64_t> slot_of_filter;
    std::vector<int4> h_segs;
    std::vector<int> h_seg_off, h_wfirst, h_active;
    std::vector<int2> h_win;                 // [n_cta] (dhi, span)
    std::vector<int> h_red_t, h_red_off;     // split templates and their zpart row ranges
    // device
    float2 *are = nullptr, *aim = nullptr, *bre = nullptr, *bim = nullptr;
    int *dly = nullptr;
    float4 *state = nullptr;
    int64_t state_det_stride = 0;
    int4 *segs = nullptr;
    int *seg_off = nullptr, *wfirst = nullptr, *active = nullptr;
    int2 *win = nullptr;
    int *red_t = nullptr, *red_off = nullptr;
    float2 *zpart = nullptr;
    int64_t zpart_pitch = 0;
    float *xbuf[2] = {nullptr, nullptr};
    int cur = 0;
    int64_t xpitch = 0, ncap = 0;
};

namespace spiir {
size_t bank_smem_bytes(const spiir_bank_s *b);
size_t bank_red_offset(const spiir_bank_s *b);
int bank_prepare(spiir_bank_s *b, int64_t ncap, cudaStream_t stream);
BankArgs bank_args(spiir_bank_s *b, float2 *z, int64_t zpitch, int64_t n);
int bank_launch_persistent(const PersistArgs &p, int S, int NL, int R, int blocks_per_sm, size_t smem,
                           cudaStream_t s);
int bank_filter(spiir_bank_s *b, const float *strain, int64_t strain_pitch, int64_t n, float2 *z,
                int64_t zpitch, cudaStream_t stream);
// Add the later delay pieces of split templates into z (after the filter launch); no-op for a
// bank without split templates.
int bank_piece_sum(spiir_bank_s *b, float2 *z, int64_t zpitch, int64_t n, cudaStream_t stream);
}
