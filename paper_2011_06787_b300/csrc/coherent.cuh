// Sky-table object and coherent-scan kernel arguments (internal).
#pragma once

#include <cstring>
#include <vector>

#include "common.cuh"

namespace spiir {

constexpr int kCohThreads = 256;                 // threads per block
constexpr int kCohQ = 2;                         // output samples per thread
constexpr int kCohMaxHalo = 1024;                // largest |Delta_I(p)| accepted
constexpr int kCohSmemTableLimit = 112 * 1024;   // table + SNR tile kept in shared memory below this


struct GroupedArgs {
    const float2 *snr;
    int64_t pitch;
    int n_templates;
    int64_t n;
    int H;
    int n_pix;
    const float4 *ent;      // [P] sorted pixels: (n0, n1, n2, plane index 1 | plane index 2 << 16)
    const uint16_t *orig;   // [P] original index of each sorted pixel
    const int4 *grp;        // [G] (plane index of detector 0, first, end, Delta_0)
    int n_grp;
    int q0, g0;             // sorted position and group of pixel 0 (tie shortcut)
    int W;                  // samples per staged plane
    float *max_stat;
    int32_t *argmax;
    float *null_stat;
    float *skymap;
    int *status;            // bounds-checked debug build only
};

// Tensor-memory scan (3 detectors): sorted pixels as in GroupedArgs, with raw offsets
// delta_I = H + Delta_I in the table entries.
struct TmemArgs {
    const float2 *snr;
    int64_t pitch;
    int n_templates;
    int64_t n;
    int H;
    int n_pix;
    const float4 *ent;      // [P] sorted pixels: (n0, n1, n2, delta_1 | delta_2 << 16)
    const uint16_t *orig;   // [P] original index of each sorted pixel
    const int4 *grp;        // [G] (unused, first, end, Delta_0)
    int n_grp;
    int q0, g0;             // sorted position and group of pixel 0
    int slice[5];           // group ranges of the four pixel slices
    int C;                  // TMEM columns used per plane (multiple of 16, at most 128)
    float *max_stat;
    int32_t *argmax;
    float *null_stat;
    float *skymap;          // NULL or [T][P][n]
    int map_vec;            // 1: n % 4 == 0 and skymap 16-byte aligned (vector stores)
    int nsub;               // templates per work item (1, 2 or 4): 128 / nsub rows each
    int mw;                 // consecutive samples per thread row: 8 (512 threads) or 16 (256)
    int sky_pix;            // pixels of the whole sky (sky-map row stride)
    int merge;              // 1: a part after the first, keep the better of the stored and the new result
};

// Per-pixel delay offsets (delta_1 | delta_2 << 16) and the pixel groups of the tensor-memory
// scan, passed as a kernel parameter when the sky is small enough: read with warp-uniform
// indices from the parameter bank, they yield tensor-memory addresses in uniform registers.
constexpr int kTmTabPix = 6400;   // with the groups, 29.7 KB: within the 32 KB of kernel parameters
constexpr int kTmTabGrp = 256;
struct TmemTab {
    uint32_t d12[kTmTabPix];
    int4 grp[kTmTabGrp];
};

int tmem_columns(int H, int mw);
bool tmem_fits(int n_pix, int n_grp, int H, int mw);

// A part of the sky for the tensor-memory scan: consecutive pixel groups (of the delay-sorted
// order) holding at most kTmTabPix pixels and kTmTabGrp groups, so that its tables travel as a
// kernel parameter.  Larger skies are cut into the fewest parts of nearly equal pixel counts and
// scanned part by part, each part keeping the better of its own and the stored (maximum, lowest
// pixel).
struct TmPart {
    int first = 0, n_pix = 0;      // sorted pixels [first, first + n_pix)
    int gfirst = 0, n_grp = 0;     // its groups (positions re-based to the part)
    int q0 = 0, g0 = 0;            // part-local sorted position and group of its lowest-index pixel
    int slice[5] = {0, 0, 0, 0, 0};
    TmemTab *tab = nullptr;        // host copy of its parameter tables
};
int tmem_templates_per_item(int64_t n, int mw);
int launch_coherent_tmem(const TmemArgs &a, const TmemTab *tab, cudaStream_t stream);

// Per-pixel entry of the general table: the two signal columns of U_s and H + Delta_I.
template <int ND>
struct __align__(16) TabEntry {
    float u[ND][2];
    short off[ND];
};

struct CohArgs {
    const float2 *snr;   // [T][n_det][pitch], entry H + k is output sample k
    int64_t pitch;
    int n_templates;
    int64_t n;
    int H;
    int n_pix;
    const void *table;   // [n_pix] entries: U_s columns and offsets H + Delta_I
    const float *u_null; // [n_pix][n_det][n_det - 2]
    float *max_stat;
    int32_t *argmax;
    float *null_stat;
    float *skymap;       // NULL or [T][n_pix][n]
    size_t tab_bytes;    // bytes of the table staged in shared memory (0: read from global)
};

}  // namespace spiir

struct spiir_sky_s {
    int n_det = 0, n_pix = 0, halo = 0;
    std::vector<unsigned char> h_table;
    size_t table_bytes = 0;
    void *table = nullptr;
    float *u_null = nullptr;
    // grouped scan (2 or 3 detectors)
    bool grouped = false;
    float4 *g_ent = nullptr;
    uint16_t *g_orig = nullptr;
    int4 *g_grp = nullptr;
    int n_grp = 0;
    int g_q0 = 0, g_g0 = 0;
    int g_W = 0;
    // launch shape of the grouped scan: threads per block and sample pairs per thread
    int scan_threads = 256, scan_pairs = 2;
    int scan_table_shared = 1;  // 1: stage the table in shared memory when it fits; 0: read it through L1
    int scan_tmem = 0;          // 1: tensor-memory scan (3 detectors, no sky map)
    int scan_tmem_param = 1;    // tensor-memory scan: 1 = group and offset tables as kernel parameters when they fit
    int scan_tmem_mw = 8;       // tensor-memory scan: samples per thread row, 8 (512 threads) or 16 (256)
    // tensor-memory scan tables (same pixel order and groups as the grouped scan)
    bool tmem_ok = false;
    float4 *t_ent = nullptr;
    std::vector<spiir::TmPart> t_parts;  // the sky in parts of the tensor-memory scan
    int4 *t_grp = nullptr;               // [G] groups with pixel positions re-based to their part
    // inputs kept to rebuild the grouped tables when the launch shape changes
    std::vector<int32_t> h_delays;
    int16_t *d_delays = nullptr;  // [P][n_det] on the device (signal-consistency gather)
    std::vector<int> rel_min, rel_max;  // [r][J]: range of Delta_J - Delta_r over the sky (on first use)
    void *pt_tab = nullptr;             // [n_det][P] per-reference point entries of the candidate scan (on first use)
    std::vector<float> h_usig, h_unull;
};

namespace spiir {
int coherent_scan(spiir_sky_s *sky, const float2 *snr, int64_t pitch, int T, int64_t n, float *max_stat,
                  int32_t *argmax, float *null_stat, float *skymap, cudaStream_t stream);
}
