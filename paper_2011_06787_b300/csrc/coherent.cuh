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
    // inputs kept to rebuild the grouped tables when the launch shape changes
    std::vector<int32_t> h_delays;
    std::vector<float> h_usig, h_unull;
};

namespace spiir {
int coherent_scan(spiir_sky_s *sky, const float2 *snr, int64_t pitch, int T, int64_t n, float *max_stat,
                  int32_t *argmax, float *null_stat, float *skymap, cudaStream_t stream);
}
